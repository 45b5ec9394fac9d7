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
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

constexpr int kMeta = 64;   // B per metadata chunk of the term-1 kernel
constexpr int kYS = 24;     // row stride (elements) of the staged Y rows (16 + 8)

// One CTA (16 warps) per (A,F) with kept B.  Shared memory (bf16 planes):
//   Cs[NP][MA][KS]   C_AF, rows alpha, K = (a,f) (row stride KS)
//   Us[NP][MB][KS]   U of the current B, rows beta, K = (a,f)
//   Vs[2][NP][MA][VS] V_AB of the current / next B (cp.async double buffer)
//   Ys[NP][YR][kYS]  Y^{BF} rows (beta,f) of the current B (NP == 2 only;
//                    prefetched while the previous B's R and Q run)
// Per-B metadata (block offsets) is resolved in chunks of kMeta B by all
// threads before the chunk's loop.
template <int NP>
__global__ void __launch_bounds__(kWarps1 * 32) k_term1_mma(DevPlan P, MixPlan X, const int* qlist, int n_list,
                                                            int MAmax, int MBmax, int KSmax, int YRmax) {
  constexpr bool kStageY = NP == 2;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 4];
  __shared__ double sacc[4];    // E (over the item) and g^V partials of the current triplet
  __shared__ int sprev;         // V pair whose g^V partials are in sacc[1..3]
  __shared__ long long m_y[kMeta], m_d[kMeta], m_v[kMeta];
  __shared__ int m_p[kMeta], m_nB[kMeta], m_mB[kMeta];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int VS = MBmax + 8;
  uint16_t* Cs = reinterpret_cast<uint16_t*>(smem);
  uint16_t* Us = Cs + (size_t)NP * MAmax * KSmax;
  uint16_t* Vs0 = Us + (size_t)NP * MBmax * KSmax;
  const size_t vbuf = (size_t)NP * MAmax * VS;
  uint16_t* Ys = Vs0 + 2 * vbuf;
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
    for (int e = threadIdx.x; e < MA * KS; e += blockDim.x) {
      const int al = e / KS, k = e - al * KS;
      const bool in = al < mA && k < KAF;
      const int a = in ? k / nF : 0, ff = in ? k - a * nF : 0;
#pragma unroll
      for (int pp = 0; pp < NP; ++pp)
        Cs[(size_t)pp * MA * KS + e] = in ? Cq[pp * cplane + ((long long)al * nA + a) * pF + ff] : (uint16_t)0;
    }
    float qacc[kQT][4];
#pragma unroll
    for (int i = 0; i < kQT; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) qacc[i][c] = 0.f;
    double g[3] = {0.0, 0.0, 0.0};
    const float* dC = reinterpret_cast<const float*>(Cq + NP * cplane);   // grad C, FP32
    const long long ncq = (long long)mA * KAF;
    const long long b0i = X.qoff[q], nbt = X.qcnt[q];
    unsigned long long fl = 0ull;
    int lastmB = -1;
    for (long long c0 = 0; c0 < nbt; c0 += kMeta) {
      const int nb = (int)min((long long)kMeta, nbt - c0);
      __syncthreads();   // previous chunk done with the metadata
      for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        const int p = X.blist[b0i + c0 + t];
        const int b = P.v_j[p];
        const int* Rb = P.v_R + 3 * p;
        const int yc = ylut_get(P, b, f, Rf[0] - Rb[0], Rf[1] - Rb[1], Rf[2] - Rb[2]);
        m_p[t] = p;
        m_y[t] = P.y_off[yc];
        m_d[t] = X.dsp_off[P.v_didx[p]];
        m_v[t] = X.vm_off[p];
        m_nB[t] = P.n_ao[P.species[b]];
        m_mB[t] = P.n_abf[P.species[b]];
      }
      __syncthreads();
      // prefetch the chunk's first B
      auto prefetch = [&](int t, int buf) {
        const int mB = m_mB[t], nB = m_nB[t];
        const int MB = rup16(mB), pB = rup16(nB);
        const uint16_t* Vg = X.Vm + m_v[t];
        uint16_t* Vd = Vs0 + buf * vbuf;
        const int vchunks = MB >> 3;                       // 16-byte chunks per V row
        for (int e = threadIdx.x; e < NP * mA * vchunks; e += blockDim.x) {
          const int pp = e / (mA * vchunks), r = e - pp * mA * vchunks;
          const int al = r / vchunks, c = r - al * vchunks;
          cp_async16(Vd + (size_t)pp * MA * VS + (size_t)al * VS + c * 8, Vg + (long long)pp * mA * MB + al * MB + c * 8);
        }
        if (kStageY && pB == 16) {
          const uint16_t* Yg = X.Ysp + m_y[t];
          const int rowsU = mB * nF;
          const int YR = YRmax;
          for (int e = threadIdx.x; e < NP * rowsU * 2; e += blockDim.x) {
            const int pp = e / (rowsU * 2), r = e - pp * rowsU * 2;
            const int row = r >> 1, c = r & 1;
            cp_async16(Ys + (size_t)pp * YR * kYS + (size_t)row * kYS + c * 8,
                       Yg + (long long)pp * rowsU * 16 + (long long)row * 16 + c * 8);
          }
        }
        cp_async_commit();
      };
      prefetch(0, 0);
      for (int t = 0; t < nb; ++t) {
        const int p = m_p[t];
        const int nB = m_nB[t], mB = m_mB[t];
        const int pB = rup16(nB), MB = rup16(mB);
        const bool ystaged = kStageY && pB == 16;
        const uint16_t* Y = X.Ysp + m_y[t];                  // [beta][f][pB] planes (global)
        const long long yplane = (long long)mB * nF * pB;
        const uint16_t* Dab = X.Dsp + m_d[t];                 // [a][pB] planes of pA x pB
        const float* V = reinterpret_cast<const float*>(X.Vm + m_v[t] + NP * mA * MB);   // V, grad V (FP32)
        const uint16_t* Vs = Vs0 + (t & 1) * vbuf;
        const int nvb = mA * mB;
        const int rowsU = mB * nF;
        cp_async_wait_all();
        __syncthreads();   // staged V (and Y) visible; previous B done with Us and sacc
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
        if (mB != lastmB) {
          // zero the Us rows beyond mB and the columns beyond KAF (never written by U)
          for (int e = threadIdx.x; e < MB * KS; e += blockDim.x) {
            const int be = e / KS, k = e - be * KS;
            if (be >= mB || k >= KAF)
#pragma unroll
              for (int pp = 0; pp < NP; ++pp) Us[(size_t)pp * MB * KS + e] = 0;
          }
          lastmB = mB;
        }
        // U[(beta,f)][a] = sum_b Y[(beta,f)][b] D_AB[a][b]  ->  Us[beta][a*nF + f]
        {
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
              if (ystaged) {
                // rows beyond rowsU read stale staged data; their results are discarded
#pragma unroll
                for (int pp = 0; pp < NP; ++pp)
                  ldm_x4(af[pp], Ys + (size_t)pp * YRmax * kYS + (size_t)(mt * 16 + (lane & 15)) * kYS + ((lane >> 4) << 3));
              } else {
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                  const int r = mt * 16 + gid + ((h & 1) ? 8 : 0);
                  const int kc = k0 + 2 * tig + ((h & 2) ? 8 : 0);
#pragma unroll
                  for (int pp = 0; pp < NP; ++pp)
                    af[pp][h] = r < rowsU ? *reinterpret_cast<const uint32_t*>(Y + pp * yplane + (long long)r * pB + kc) : 0u;
                }
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
        __syncthreads();   // Us ready; Ys and the other V buffer free
        if (t + 1 < nb) prefetch(t + 1, (t + 1) & 1);
        // R_t = C_AF . U^T (M = alpha, N = beta, K = (a,f)); dotted with V and grad V
        float evf[4] = {0.f, 0.f, 0.f, 0.f};
        {
          const int NTR = MB >> 3;
          const int nt_tiles = MT * NTR;
          for (int tt = warp; tt < nt_tiles; tt += kWarps1) {
            const int mt = tt / NTR, nt = tt - mt * NTR;
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
#pragma unroll
        for (int i = 0; i < kQT; ++i) {
          const int tt = warp + i * kWarps1;
          if (tt >= MT * NTq) continue;
          const int mt = tt / NTq, nt = tt - mt * NTq;
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
        // flush the FP32 run of Q into the FP64 gradient dot
        const long long bi = c0 + t;
        if ((bi % kFlush) == kFlush - 1 || bi + 1 == nbt) {
          float gf[3] = {0.f, 0.f, 0.f};
#pragma unroll
          for (int i = 0; i < kQT; ++i) {
            const int tt = warp + i * kWarps1;
            if (tt >= MT * NTq) continue;
            const int mt = tt / NTq, nt = tt - mt * NTq;
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
// Phase 1: one CTA per kept (A,B) pair of the second product (slot s of the
// pair list).  Shared memory (bf16 planes, row stride KZ = n_ao(A)*pB + 8):
//   Yb[NP][MB][KZ]  Y^{BA} as [beta][(a,b)]         (b padded to pB)
//   Ya[NP][MA][KZ]  Y^{AB} transposed to [alpha][(a,b)]
// R2^T[beta][alpha] = sum_{(a,b)} Yb[beta][(a,b)] Ya[alpha][(a,b)], dotted with V, grad V;
// Z[alpha][(a,b)] = sum_beta V[alpha][beta] Yb[beta][(a,b)] -> Z store of slot s as
// NP planes [(alpha,a)][pB].
template <int NP>
__global__ void __launch_bounds__(kWarps * 32) k_term2_pairs(DevPlan P, MixPlan X, const int* list, int n_list,
                                                             int MAmax, int KZmax, long long zblk, int zrows) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32 * 4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  uint16_t* Yb = reinterpret_cast<uint16_t*>(smem);
  uint16_t* Ya = Yb + (size_t)NP * MAmax * KZmax;
  for (int kk = blockIdx.x; kk < n_list; kk += gridDim.x) {
    const int p = list[kk];
    const int A = P.v_home[p], b = P.v_j[p];
    const int* Rb = P.v_R + 3 * p;
    const int sA = P.species[A], sB = P.species[b];
    const int nA = P.n_ao[sA], nB = P.n_ao[sB], mA = P.n_abf[sA], mB = P.n_abf[sB];
    const int pA = rup16(nA), pB = rup16(nB);
    const int MA = rup16(mA), MB = rup16(mB);
    const int NAB = nA * pB, KZ = NAB + 8;
    const int y1 = ylut_get(P, A, b, Rb[0], Rb[1], Rb[2]);
    const int y2 = ylut_get(P, b, A, -Rb[0], -Rb[1], -Rb[2]);
    const uint16_t* Yab = X.Ysp + P.y_off[y1];   // [alpha][b][pA]
    const uint16_t* Yba = X.Ysp + P.y_off[y2];   // [beta][a][pB]
    const long long pl_ab = (long long)mA * nB * pA, pl_ba = (long long)mB * nA * pB;
    const uint16_t* Vp = X.Vm + X.vm_off[p];
    const float* V = reinterpret_cast<const float*>(Vp + NP * mA * MB);
    const int nvb = mA * mB;
    __syncthreads();
    // stage Y^{BA} rows (contiguous copy) and Y^{AB} transposed
    for (int e = threadIdx.x; e < MB * KZ; e += blockDim.x) {
      const int be = e / KZ, c = e - be * KZ;
      const bool in = be < mB && c < NAB;
#pragma unroll
      for (int pp = 0; pp < NP; ++pp) Yb[(size_t)pp * MB * KZ + e] = in ? Yba[pp * pl_ba + (long long)be * NAB + c] : (uint16_t)0;
    }
    for (int e = threadIdx.x; e < MA * KZ; e += blockDim.x) {
      const int al = e / KZ, c = e - al * KZ;
      const int a = c / pB, bb = c - a * pB;
      const bool in = al < mA && c < NAB && bb < nB;
#pragma unroll
      for (int pp = 0; pp < NP; ++pp)
        Ya[(size_t)pp * MA * KZ + e] = in ? Yab[pp * pl_ab + ((long long)al * nB + bb) * pA + a] : (uint16_t)0;
    }
    __syncthreads();
    // R2^T (M = beta, N = alpha, K = (a,b))
    float evf[4] = {0.f, 0.f, 0.f, 0.f};
    {
      const int MT = MB >> 4, NT = MA >> 3;
      for (int t = warp; t < MT * NT; t += kWarps) {
        const int mt = t / NT, nt = t - mt * NT;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k0 = 0; k0 < NAB; k0 += 16) {
          uint32_t af[NP][4], bf[NP][2];
#pragma unroll
          for (int pp = 0; pp < NP; ++pp) {
            ldm_x4(af[pp], Yb + (size_t)pp * MB * KZ + (size_t)(mt * 16 + (lane & 15)) * KZ + k0 + ((lane >> 4) << 3));
            ldm_x2(bf[pp], Ya + (size_t)pp * MA * KZ + (size_t)(nt * 8 + (lane & 7)) * KZ + k0 + (((lane >> 3) & 1) << 3));
          }
          mma_split<NP>(acc, af, bf);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int be = mt * 16 + gid + ((c & 2) ? 8 : 0);
          const int al = nt * 8 + 2 * tig + (c & 1);
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
    // Z (M = alpha, N = (a,b), K = beta) -> Z store
    {
      uint16_t* Zo = X.Zst + (long long)kk * zblk;
      const long long zpl = (long long)zrows * pB;
      const int MT = MA >> 4, NT = NAB >> 3;
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
#pragma unroll
          for (int pp = 0; pp < NP; ++pp)
            ldm_x2_trans(bf[pp], Yb + (size_t)pp * MB * KZ + (size_t)(k0 + (lane & 15)) * KZ + nt * 8);
          mma_split<NP>(acc, af, bf);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int al = mt * 16 + gid + (h ? 8 : 0);
          const int col = nt * 8 + 2 * tig;          // even: (a, bb) and (a, bb+1)
          if (al < mA) {
            const int a = col / pB, bb = col - a * pB;
            uint16_t p0[NP], p1[NP];
            split_f<NP>(acc[2 * h], p0);
            split_f<NP>(acc[2 * h + 1], p1);
#pragma unroll
            for (int pp = 0; pp < NP; ++pp)
              *reinterpret_cast<uint32_t*>(Zo + pp * zpl + (long long)(al * nA + a) * pB + bb) = pack2(p0[pp], p1[pp]);
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
      atomicAdd(&P.acc[ACC_F2], 4.0 * mA * mB * nA * nB);
    }
  }
}

// Phase 2: Q2^{AF}[(alpha,a)][f] = sum_{B} sum_b Z^{AB}[(alpha,a)][b] D_FB[f][b]
// as one GEMM per home atom A (K = (B, b) over its pairs of the second
// product), dotted with grad C_AF.  CTA = (A, 4 C slots F, 128 rows); each
// warp owns one 16-row tile and the 4 x 2 column tiles of the 4 F.  The D
// blocks of each chunk of pairs are resolved into shared memory first.
constexpr int kQ2Meta = 64;
template <int NP>
__global__ void __launch_bounds__(kWarps * 32, 2) k_q2_gemm(DevPlan P, MixPlan X, const int* list,
                                                            const long long* slot0, int n_slots, int FC, int MC,
                                                            long long zblk, int zrows) {
  __shared__ long long m_d[kQ2Meta][4];
  __shared__ int m_pB[kQ2Meta], m_nB[kQ2Meta];
  __shared__ double sg[4][3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int A = blockIdx.x / (FC * MC);
  const int rem = blockIdx.x - A * FC * MC;
  const int fc = rem / MC, mc = rem - fc * MC;
  const int sA = P.species[A];
  const int nA = P.n_ao[sA], mA = P.n_abf[sA];
  const int rows = mA * nA;
  const int q0 = P.c_ptr[A], nq = P.c_ptr[A + 1] - q0;
  if (fc * 4 >= nq || mc * 128 >= rows) return;
  const int mt = mc * 8 + warp;
  const bool active = mt * 16 < rows;
  int qf[4], nF[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int j = fc * 4 + i;
    qf[i] = (j < nq && P.c_keep[q0 + j]) ? q0 + j : -1;
    nF[i] = qf[i] >= 0 ? P.n_ao[P.species[P.c_j[qf[i]]]] : 0;
  }
  if (threadIdx.x < 12) sg[threadIdx.x / 3][threadIdx.x % 3] = 0.0;
  const long long s0 = slot0[P.v_ptr[A]];
  const long long s1 = A + 1 < P.N ? slot0[P.v_ptr[A + 1]] : (long long)n_slots;
  float acc[4][2][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[i][n][c] = 0.f;
  unsigned long long fl = 0ull;
  int run = 0;
  for (long long c0 = s0; c0 < s1; c0 += kQ2Meta) {
    const int nb = (int)min((long long)kQ2Meta, s1 - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < nb * 4; e += blockDim.x) {
      const int t = e >> 2, i = e & 3;
      const int p = list[c0 + t];
      const int b = P.v_j[p];
      const int* Rb = P.v_R + 3 * p;
      long long doff = -1;
      if (qf[i] >= 0) {
        const int* Rf = P.c_R + 3 * qf[i];
        const int d = dlut_get(P, P.c_j[qf[i]], b, Rb[0] - Rf[0], Rb[1] - Rf[1], Rb[2] - Rf[2]);
        if (d >= 0 && P.Dkept[d] != 0.0) doff = X.dsp_off[d];
      }
      m_d[t][i] = doff;
      if (i == 0) {
        m_nB[t] = P.n_ao[P.species[b]];
        m_pB[t] = rup16(m_nB[t]);
      }
    }
    __syncthreads();
    if (mc == 0 && threadIdx.x == 0)
      for (int t = 0; t < nb; ++t)
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (m_d[t][i] >= 0) fl += 2ull * mA * nA * m_nB[t] * nF[i];
    for (int t = 0; t < nb; ++t) {
      const int pB = m_pB[t];
      if (active) {
        const uint16_t* Zp = X.Zst + (c0 + t) * zblk;
        const long long zpl = (long long)zrows * pB;
        for (int k0 = 0; k0 < pB; k0 += 16) {
          uint32_t af[NP][4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int r = mt * 16 + gid + ((h & 1) ? 8 : 0);
            const int kc = k0 + 2 * tig + ((h & 2) ? 8 : 0);
#pragma unroll
            for (int pp = 0; pp < NP; ++pp)
              af[pp][h] = r < rows ? *reinterpret_cast<const uint32_t*>(Zp + pp * zpl + (long long)r * pB + kc) : 0u;
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const long long doff = m_d[t][i];
            if (doff < 0) continue;
            const int pF = rup16(nF[i]);
            const uint16_t* Dfb = X.Dsp + doff;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
              if (nt * 8 >= pF) continue;
              uint32_t bf[NP][2];
#pragma unroll
              for (int pp = 0; pp < NP; ++pp) {
                const uint16_t* Db = Dfb + pp * pF * pB + (nt * 8 + gid) * pB + k0 + 2 * tig;
                bf[pp][0] = *reinterpret_cast<const uint32_t*>(Db);
                bf[pp][1] = *reinterpret_cast<const uint32_t*>(Db + 8);
              }
              mma_split<NP>(acc[i][nt], af, bf);
            }
          }
        }
      }
      // flush the FP32 run into the FP64 gradient dots (shared accumulators)
      if (++run == 32 || c0 + t + 1 == s1) {
        run = 0;
        if (active) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float gf[3] = {0.f, 0.f, 0.f};
            if (qf[i] >= 0) {
              const int pF = rup16(nF[i]);
              const int KAF = nA * nF[i];
              const long long ncq = (long long)mA * KAF;
              const float* dC = reinterpret_cast<const float*>(X.Cm + X.cm_off[qf[i]] + (long long)NP * rows * pF);
#pragma unroll
              for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  const int r = mt * 16 + gid + ((c & 2) ? 8 : 0);
                  const int ff = nt * 8 + 2 * tig + (c & 1);
                  if (r < rows && ff < nF[i]) {
                    const int al = r / nA, a = r - al * nA;
                    const long long o = (long long)al * KAF + a * nF[i] + ff;
                    const float v = acc[i][nt][c];
                    gf[0] = fmaf(dC[o], v, gf[0]);
                    gf[1] = fmaf(dC[ncq + o], v, gf[1]);
                    gf[2] = fmaf(dC[2 * ncq + o], v, gf[2]);
                  }
                  acc[i][nt][c] = 0.f;
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float w = warp_sum_f(gf[c]);
              if (lane == 0 && w != 0.f) atomicAdd(&sg[i][c], (double)w);
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    const int i = threadIdx.x / 3, c = threadIdx.x % 3;
    if (qf[i] >= 0 && sg[i][c] != 0.0) atomicAdd(&P.gC[3 * qf[i] + c], -2.0 * sg[i][c]);
  }
  if (threadIdx.x == 0 && fl) atomicAdd(&P.acc[ACC_F2], (double)fl);
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

size_t term1_mma_smem(int np, int MAmax, int MBmax, int KSmax, int YRmax) {
  size_t e = (size_t)np * (MAmax * KSmax + MBmax * KSmax + 2 * MAmax * (MBmax + 8));
  if (np == 2) e += (size_t)np * YRmax * kYS;
  return e * sizeof(uint16_t);
}

size_t term2_mma_smem(int np, int MAmax, int KZmax) {
  return (size_t)np * 2 * MAmax * KZmax * sizeof(uint16_t);
}

cudaError_t set_mixed_smem_limits(int np, size_t t1, size_t t2) {
  cudaError_t e;
  if (np == 2) {
    e = cudaFuncSetAttribute(k_term1_mma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t1);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_term2_pairs<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t2);
  }
  e = cudaFuncSetAttribute(k_term1_mma<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t1);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_term2_pairs<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t2);
}

cudaError_t launch_term1_mma(const DevPlan& P, const MixPlan& X, int np, const int* qlist, int n, int MAmax, int MBmax,
                             int KSmax, int YRmax, size_t smem, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  ++g_mix_launches;
  if (np == 2)
    k_term1_mma<2><<<grid_for(n, 152 * 16), kWarps1 * 32, smem, s>>>(P, X, qlist, n, MAmax, MBmax, KSmax, YRmax);
  else
    k_term1_mma<3><<<grid_for(n, 152 * 16), kWarps1 * 32, smem, s>>>(P, X, qlist, n, MAmax, MBmax, KSmax, YRmax);
  return cudaGetLastError();
}

cudaError_t launch_term2_mma(const DevPlan& P, const MixPlan& X, int np, const int* list, const long long* slot0,
                             int n, int MAmax, int KZmax, long long zblk, int zrows, int FC, int MC, size_t smem,
                             cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  g_mix_launches += 2;
  if (np == 2) {
    k_term2_pairs<2><<<grid_for(n, 152 * 32), kWarps * 32, smem, s>>>(P, X, list, n, MAmax, KZmax, zblk, zrows);
    k_q2_gemm<2><<<P.N * FC * MC, kWarps * 32, 0, s>>>(P, X, list, slot0, n, FC, MC, zblk, zrows);
  } else {
    k_term2_pairs<3><<<grid_for(n, 152 * 32), kWarps * 32, smem, s>>>(P, X, list, n, MAmax, KZmax, zblk, zrows);
    k_q2_gemm<3><<<P.N * FC * MC, kWarps * 32, 0, s>>>(P, X, list, slot0, n, FC, MC, zblk, zrows);
  }
  return cudaGetLastError();
}

}  // namespace hfx
