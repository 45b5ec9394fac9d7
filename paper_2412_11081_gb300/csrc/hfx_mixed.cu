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

#include <atomic>
#include <cstdint>

#include "hfx_accum.cuh"
#include "hfx_device.cuh"
#include "hfx_model.cuh"

namespace hfx {
namespace {

using namespace dev;

constexpr int kWarps1 = 16;     // warps per CTA of the term-1 kernel
constexpr int kWarps = 8;       // warps per CTA of the other mixed kernels
constexpr int kQT = 16;         // Q accumulator tiles per warp (term 1)
constexpr int kFlush = 8;       // B per FP32 run of the Q accumulators
std::atomic<long long> g_mix_launches{0};

// Element offset of (row r, column c < 16) inside a tile stored in the
// K-major core-matrix order of the tensor cores: 8-row x 8-column core
// matrices (16 bytes per row), the two column halves 64 elements apart and
// 8-row groups 128 elements apart.  D piece blocks (16 x 16) and the Z store
// (128-row tiles) use it, so a tile is copied to shared memory as one block.
__device__ __forceinline__ int tix(int r, int c) { return ((r >> 3) << 7) + ((c >> 3) << 6) + ((r & 7) << 3) + (c & 7); }

// Element (row r, column k) of a tile of K columns (K a multiple of 8) in the
// tensor cores' K-major core-matrix order: 8-row groups of K / 8 core matrices
// (8 rows x 16 bytes each), the core matrices of a group consecutive.
__device__ __forceinline__ long long cmx(int r, int k, int K) {
  return (long long)(r >> 3) * 8 * K + ((k >> 3) << 6) + ((r & 7) << 3) + (k & 7);
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
      for (int p = 0; p < NP; ++p) out[p * pa * pb + tix(a, b)] = pc[p];
    }
  }
}

// ------------------------------------------------------------------ pieces
// C pair q: NP bf16 pieces of C[(alpha,a)][f] in 128-row tiles of the
// tensor cores' core-matrix order ([tile][piece][128 x 16], f padded to 16),
// then grad C in FP32 ([3][(alpha,a)][f]).
template <int NP>
__global__ void k_cpieces(DevPlan P, MixPlan X) {
  for (int q = blockIdx.x; q < P.nC; q += gridDim.x) {
    if (!P.c_keep[q]) continue;
    const int A = P.c_home[q], f = P.c_j[q];
    const int sA = P.species[A], sF = P.species[f];
    const int rows = P.n_abf[sA] * P.n_ao[sA], nF = P.n_ao[sF];
    const int nt = (rows + 127) >> 7;
    // C and grad C evaluated in FP32 from the block model (scalars of k_cnorm)
    float scf[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) scf[k] = (float)P.c_sc[8 * (long long)q + k];
    const long long go = P.G_off[sA * P.S + sF];
    uint16_t* out = X.Cm + X.cm_off[q];
    for (int e = threadIdx.x; e < nt * 128 * 16; e += blockDim.x) {
      const int r = e >> 4, c = e & 15;
      uint16_t pc[NP];
      split_f<NP>((r < rows && c < nF) ? model::c_value_f(P, scf, go, r * nF + c, 0) : 0.f, pc);
#pragma unroll
      for (int p = 0; p < NP; ++p) out[((r >> 7) * NP + p) * 2048 + tix(r & 127, c)] = pc[p];
    }
    // grad C in FP32, three components in the tile order of gc_off (written in storage order)
    float* g = reinterpret_cast<float*>(out + NP * nt * 2048);
    for (int w = threadIdx.x; w < 3 * nt * 2048; w += blockDim.x) {
      const int c = w / (nt * 2048), wi = w - c * nt * 2048;
      const int r = ((wi >> 11) << 7) + ((wi >> 2) & 127), ff = (((wi >> 9) & 3) << 2) + (wi & 3);
      g[w] = (r < rows && ff < nF) ? model::c_value_f(P, scf, go, r * nF + ff, c + 1) : 0.f;
    }
  }
}

// needed V pair p: NP bf16 planes of V[alpha][rup16(n_abf(B))] then V, grad V (FP32),
// evaluated from the block model (V = M h, grad V = M g) without an FP64 store.
template <int NP>
__global__ void k_vpieces(DevPlan P, MixPlan X, const int* list, int n_list) {
  for (int k = blockIdx.x; k < n_list; k += gridDim.x) {
    const int p = list[k];
    const int sA = P.species[P.v_home[p]], sB = P.species[P.v_j[p]];
    const int mA = P.n_abf[sA], mB = P.n_abf[sB];
    const int MB = rup16(mB);
    double h, g[3];
    model::v_pair(P, p, h, g);
    const float hf = (float)h, g0 = (float)g[0], g1 = (float)g[1], g2 = (float)g[2];
    const float* M = P.Mf + P.M_off[sA * P.S + sB];   // FP32 products, as k_vstores
    uint16_t* out = X.Vm + X.vm_off[p];
    for (int e = threadIdx.x; e < mA * MB; e += blockDim.x) {
      const int al = e / MB, be = e - al * MB;
      uint16_t pc[NP];
      split_f<NP>(be < mB ? M[al * mB + be] * hf : 0.f, pc);
#pragma unroll
      for (int pp = 0; pp < NP; ++pp) out[pp * mA * MB + e] = pc[pp];
    }
    float* v32 = reinterpret_cast<float*>(out + NP * mA * MB);
    const int n = mA * mB;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const float m = M[e];
      v32[e] = m * hf;
      v32[n + e] = m * g0;
      v32[2 * n + e] = m * g1;
      v32[3 * n + e] = m * g2;
    }
  }
}

// --------------------------------------------------- term-1 transposed lists
// Per home atom A: for every C slot of A, the V pairs (A,B) whose item list
// keeps it, in V-pair order (deterministic).
// (A,F) view of the first product's kept triplets: one warp per C pair
// (A,F) = q, its lanes test 32 V pairs of A at a time.  Phase 0 counts the
// kept B (qcnt), phase 1 writes them in V-pair order from qoff (ballot and
// prefix count keep the order).
__global__ void k_t1_lists(DevPlan P, MixPlan X, int phase) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int q = blockIdx.x * wpb + (threadIdx.x >> 5); q < P.nC; q += gridDim.x * wpb) {
    const int A = P.c_home[q], s = q - P.c_ptr[A];
    const int p0 = P.v_ptr[A], p1 = P.v_ptr[A + 1];
    long long o = phase ? X.qoff[q] : 0;
    int cnt = 0;
    for (int pb = p0; pb < p1; pb += 32) {
      const int p = pb + lane;
      const bool kept = p < p1 && ((P.v_mask[(size_t)p * kMaskWords + (s >> 5)] >> (s & 31)) & 1u);
      const unsigned bal = __ballot_sync(0xffffffffu, kept);
      if (phase && kept) X.blist[o + __popc(bal & ((1u << lane) - 1u))] = p;
      o += __popc(bal);
      cnt += __popc(bal);
    }
    if (!phase && lane == 0) X.qcnt[q] = cnt;
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
    const uint16_t* Cq = X.Cm + X.cm_off[q];
    const int ctiles = (mA * nA + 127) >> 7;
    for (int e = threadIdx.x; e < MA * KS; e += blockDim.x) {
      const int al = e / KS, k = e - al * KS;
      const bool in = al < mA && k < KAF;
      const int a = in ? k / nF : 0, ff = in ? k - a * nF : 0;
      const int r = al * nA + a;
#pragma unroll
      for (int pp = 0; pp < NP; ++pp)
        Cs[(size_t)pp * MA * KS + e] = in ? Cq[((r >> 7) * NP + pp) * 2048 + tix(r & 127, ff)] : (uint16_t)0;
    }
    float qacc[kQT][4];
#pragma unroll
    for (int i = 0; i < kQT; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) qacc[i][c] = 0.f;
    double g[3] = {0.0, 0.0, 0.0};
    const float* dC = reinterpret_cast<const float*>(Cq + (long long)NP * ctiles * 2048);   // grad C, FP32
    const long long ncq = (long long)ctiles * 2048;   // floats per grad C component
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
            dev::add_gV(P, 3 * sprev + 0, -sacc[1]);
            dev::add_gV(P, 3 * sprev + 1, -sacc[2]);
            dev::add_gV(P, 3 * sprev + 2, -sacc[3]);
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
              for (int nt = 0; nt < 4; nt += 2) {
                if (nt >= NTU) break;
                uint32_t bf0[NP][2], bf1[NP][2];
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) {
                  const uint16_t* Db = Dab + pp * 256 + tix(nt * 8 + gid, 2 * tig);
                  bf0[pp][0] = *reinterpret_cast<const uint32_t*>(Db);
                  bf0[pp][1] = *reinterpret_cast<const uint32_t*>(Db + 64);
                  bf1[pp][0] = *reinterpret_cast<const uint32_t*>(Db + 128);
                  bf1[pp][1] = *reinterpret_cast<const uint32_t*>(Db + 192);
                }
                mma_split2<NP>(acc[nt], af, bf0, acc[nt + 1], af, bf1);
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
        // R_t = C_AF . U^T (M = alpha, N = beta, K = (a,f)); dotted with V and grad V.
        // Warp -> one alpha tile (A fragments reused) and up to two beta tiles
        // (their product chains interleaved).
        float evf[4] = {0.f, 0.f, 0.f, 0.f};
        {
          const int NTR = MB >> 3;
          const int wpm = kWarps1 / MT;              // warps per alpha tile
          const int mt = warp % MT, w0 = warp / MT;
          if (w0 < wpm) {
            for (int nt0 = w0; nt0 < NTR; nt0 += 2 * wpm) {
              const int nt1 = nt0 + wpm;
              const bool two = nt1 < NTR;
              float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};
              for (int k0 = 0; k0 < KP; k0 += 16) {
                uint32_t af[NP][4], bf0[NP][2], bf1[NP][2];
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) {
                  ldm_x4(af[pp], Cs + (size_t)pp * MA * KS + (size_t)(mt * 16 + (lane & 15)) * KS + k0 + ((lane >> 4) << 3));
                  ldm_x2(bf0[pp], Us + (size_t)pp * MB * KS + (size_t)(nt0 * 8 + (lane & 7)) * KS + k0 + (((lane >> 3) & 1) << 3));
                  ldm_x2(bf1[pp], Us + (size_t)pp * MB * KS + (size_t)((two ? nt1 : nt0) * 8 + (lane & 7)) * KS + k0 +
                                      (((lane >> 3) & 1) << 3));
                }
                mma_split2<NP>(acc0, af, bf0, acc1, af, bf1);
              }
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                if (h == 1 && !two) break;
                const int nt = h ? nt1 : nt0;
                const float* acc = h ? acc1 : acc0;
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
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float w = warp_sum_f(evf[c]);
          if (lane == 0) {
            if (P.fxC)   // deterministic plan: straight into the exact cells
              (c == 0) ? dev::add_E(P, -(double)w) : dev::add_gV(P, 3 * p + c - 1, -(double)w);
            else
              atomicAdd(&sacc[c], (double)w);
          }
        }
        // Q += V_AB . U (M = alpha, N = (a,f), K = beta).  Warp -> one alpha tile
        // and the (a,f) tiles nt = w0 + i * wpm; tiles i, i + 1 interleaved.
        {
          const int wpm = kWarps1 / MT;
          const int mt = warp % MT, w0 = warp / MT;
          if (w0 < wpm) {
            for (int k0 = 0; k0 < MB; k0 += 16) {
              uint32_t af[NP][4];
#pragma unroll
              for (int pp = 0; pp < NP; ++pp)
                ldm_x4(af[pp], Vs + (size_t)pp * MA * VS + (size_t)(mt * 16 + (lane & 15)) * VS + k0 + ((lane >> 4) << 3));
#pragma unroll
              for (int i = 0; i < kQT; i += 2) {
                const int nt0 = w0 + i * wpm, nt1 = w0 + (i + 1) * wpm;
                if (nt0 >= NTq) continue;
                const bool two = nt1 < NTq;
                uint32_t bf0[NP][2], bf1[NP][2];
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) {
                  ldm_x2_trans(bf0[pp], Us + (size_t)pp * MB * KS + (size_t)(k0 + (lane & 15)) * KS + nt0 * 8);
                  ldm_x2_trans(bf1[pp], Us + (size_t)pp * MB * KS + (size_t)(k0 + (lane & 15)) * KS + (two ? nt1 : nt0) * 8);
                }
                if (two) mma_split2<NP>(qacc[i], af, bf0, qacc[i + 1], af, bf1);
                else mma_split<NP>(qacc[i], af, bf0);
              }
            }
          }
        }
        // flush the FP32 run of Q into the FP64 gradient dot
        const long long bi = c0 + t;
        if ((bi % kFlush) == kFlush - 1 || bi + 1 == nbt) {
          float gf[3] = {0.f, 0.f, 0.f};
          const int wpm = kWarps1 / MT;
          const int mt = warp % MT, w0 = warp / MT;
#pragma unroll
          for (int i = 0; i < kQT; ++i) {
            const int nt = w0 + i * wpm;
            if (w0 >= wpm || nt >= NTq) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int al = mt * 16 + gid + ((c & 2) ? 8 : 0);
              const int n = nt * 8 + 2 * tig + (c & 1);
              if (al < mA && n < KAF) {
                const int a = n / nF;
                const int o = gc_off(al * nA + a, n - a * nF);
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
      dev::add_gC(P, 3 * q + 0, -2.0 * g[0]);
      dev::add_gC(P, 3 * q + 1, -2.0 * g[1]);
      dev::add_gC(P, 3 * q + 2, -2.0 * g[2]);
      if (sprev >= 0) {
        dev::add_gV(P, 3 * sprev + 0, -sacc[1]);
        dev::add_gV(P, 3 * sprev + 1, -sacc[2]);
        dev::add_gV(P, 3 * sprev + 2, -sacc[3]);
      }
      dev::add_E(P, -sacc[0]);
      atomicAdd(&P.acc[ACC_F1], (double)fl);
    }
  }
}

// ------------------------------------------------------------------ term 2
// Phase 1: one CTA per kept (A,B) pair of the second product (slot s of the
// pair list).  Shared memory (bf16 planes, row stride KZ = n_ao(A)*pB + 8):
//   Yb[NP][MB][KZ]  Y^{BA} as [beta][(a,b)]         (b padded to pB)
//   Ya[NP][MA][KZ]  Y^{AB} as [alpha][(a,b)], from the transposed store the Y build writes
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
    constexpr int pB = 16;   // the split path holds n_ao <= 16
    const int MA = rup16(mA), MB = rup16(mB);
    const int NAB = nA * pB, KZ = NAB + 8;
    const int y1 = ylut_get(P, A, b, Rb[0], Rb[1], Rb[2]);
    const int y2 = ylut_get(P, b, A, -Rb[0], -Rb[1], -Rb[2]);
    const uint16_t* YabT = X.YspT + X.y_idx[y1] * X.yT_blk;   // Y^{AB} transposed: [alpha][a][pB]
    const uint16_t* Yba = X.Ysp + P.y_off[y2];                  // [beta][a][pB]
    const long long pl_abT = X.yT_blk / NP, pl_ba = (long long)mB * nA * pB;
    const uint16_t* Vp = X.Vm + X.vm_off[p];
    const float* V = reinterpret_cast<const float*>(Vp + NP * mA * MB);
    const int nvb = mA * mB;
    __syncthreads();
    // stage the rows [(a,b)] of Y^{BA} (by beta) and of the transposed Y^{AB}
    // (by alpha) with 16-byte copies (rows NAB long, shared-memory stride KZ;
    // rows past n_abf zero, columns past NAB never read)
    {
      const int nch = NAB >> 3;   // 16-byte chunks per row (2 n_ao(A) <= 32: one lane each)
      for (int rr = warp; rr < MB + MA; rr += kWarps) {
        const bool isA = rr >= MB;
        const int row = isA ? rr - MB : rr;
        const bool in = row < (isA ? mA : mB);
        if (lane < nch) {
#pragma unroll
          for (int pp = 0; pp < NP; ++pp) {
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (in)
              v = *reinterpret_cast<const uint4*>((isA ? YabT + pp * pl_abT : Yba + pp * pl_ba) + (long long)row * NAB + 8 * lane);
            uint16_t* dst = isA ? Ya + (size_t)pp * MA * KZ : Yb + (size_t)pp * MB * KZ;
            *reinterpret_cast<uint4*>(dst + (size_t)row * KZ + 8 * lane) = v;
          }
        }
      }
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
    // Z (M = alpha, N = (a,b), K = beta) -> Z store, 128-row tiles of rows (alpha,a)
    {
      uint16_t* Zo = X.Zst + (long long)kk * zblk;
      const int MT = MA >> 4, NT = NAB >> 3;
      // With n_abf(B) <= 64 (four k steps) a warp keeps one row tile mt and
      // its V fragments in registers across the column tiles it takes;
      // larger n_abf(B) reload them per tile.
      const bool keepA = MB <= 64;
      const int nslot = keepA ? kWarps / MT : 1;
      const int t0 = keepA ? (warp < nslot * MT ? (warp % MT) * NT + warp / MT : MT * NT) : warp;
      const int tstep = keepA ? nslot : kWarps;
      uint32_t ak[4][NP][4];
      int mt_loaded = -1;
      for (int t = t0; t < (keepA ? ((t0 / NT) + 1) * NT : MT * NT); t += tstep) {
        const int mt = t / NT, nt = t - mt * NT;
        if (keepA && mt != mt_loaded) {
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int al = mt * 16 + gid + ((h & 1) ? 8 : 0);
              const int kc = ks * 16 + 2 * tig + ((h & 2) ? 8 : 0);
#pragma unroll
              for (int pp = 0; pp < NP; ++pp)
                ak[ks][pp][h] = (al < mA && kc < MB) ? *reinterpret_cast<const uint32_t*>(Vp + pp * mA * MB + al * MB + kc) : 0u;
            }
          mt_loaded = mt;
        }
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (keepA) {
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            if (ks * 16 >= MB) break;
            uint32_t bf[NP][2];
#pragma unroll
            for (int pp = 0; pp < NP; ++pp)
              ldm_x2_trans(bf[pp], Yb + (size_t)pp * MB * KZ + (size_t)(ks * 16 + (lane & 15)) * KZ + nt * 8);
            mma_split<NP>(acc, ak[ks], bf);
          }
        } else {
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
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int al = mt * 16 + gid + (h ? 8 : 0);
          const int col = nt * 8 + 2 * tig;          // even: (a, bb) and (a, bb+1)
          if (al < mA) {
            const int a = col >> 4, bb = col & 15;
            uint16_t p0[NP], p1[NP];
            split_f<NP>(acc[2 * h], p0);
            split_f<NP>(acc[2 * h + 1], p1);
            const int r = al * nA + a;
#pragma unroll
            for (int pp = 0; pp < NP; ++pp)
              *reinterpret_cast<uint32_t*>(Zo + ((long long)(r >> 7) * NP + pp) * 2048 + tix(r & 127, bb)) =
                  pack2(p0[pp], p1[pp]);
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
      dev::add_E(P, -ev[0]);
      dev::add_gV(P, 3 * p + 0, -ev[1]);
      dev::add_gV(P, 3 * p + 1, -ev[2]);
      dev::add_gV(P, 3 * p + 2, -ev[3]);
      atomicAdd(&P.acc[ACC_F2], 4.0 * mA * mB * nA * nB);
    }
  }
}

// ------------------------------------------------------------ tcgen05 Q2 GEMM
// Same product as k_q2_gemm on the 5th-generation tensor cores: per CTA
// (home atom A, 8 C slots F, 128 rows (alpha,a)), D[row][(F,f)] +=
// Z^{AB}[row][b] D_FB[f][b] over the pairs (A,B) of the second product, one
// k16 step per pair and all bf16 piece products into one FP32 accumulator in
// tensor memory (128 lanes x 128 columns).  Operands are staged by cp.async in
// the K-major no-swizzle core-matrix layout (8 rows x 16 bytes per core
// matrix; LBO = 128 B between the two K halves, SBO = 256 B between 8-row
// groups) through a 4-stage ring; thread 0 issues the MMAs and commits each
// stage to an mbarrier.  Every 32 pairs the accumulator is read back
// (tcgen05.ld) and dotted with grad C_AF into FP64.  Every wait is bounded;
// on timeout the CTA sets *err and stops.
namespace umma {

constexpr int kStages = 4;
constexpr uint32_t kMixTryNs = kTryNs;   // suspend hint of the pipeline waits
constexpr int kTileElems = 128 * 16;     // bf16 elements of one 128 x 16 operand tile (one piece)
constexpr int kMetaPairs = 1024;         // pairs per CTA segment (metadata in shared memory)

// K-major operand tiles: K-adjacent core matrices 128 bytes apart, 8-row groups 256 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) { return sdesc2(saddr, 128, 256); }

// Four 512-byte rows r0..r3 of the D piece store (tensor map of DRows) to
// consecutive shared memory at sdst (128-byte aligned), completion counted in
// bytes on mbar.
__device__ __forceinline__ void gather4_rows(uint32_t sdst, const CUtensorMap* map, int r0, int r1, int r2, int r3,
                                             uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5, %6}], [%7];\n" ::"r"(sdst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(mbar)
      : "memory");
}

// Stage the B operand of one K step: D rows of the eight keys i (row md[i] +
// piece, the zero row where md[i] < 0), piece pp and key half h by lane
// 1 + 2 pp + h.
template <int NP>
__device__ __forceinline__ void stage_d(int lane, uint16_t* stB, const int* md, const CUtensorMap* map, int zrow,
                                        uint32_t mbar) {
  if (lane >= 1 && lane <= 2 * NP) {
    const int pp = (lane - 1) >> 1, h = (lane - 1) & 1;
    int r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int d = md[4 * h + j];
      r[j] = d >= 0 ? d + pp : zrow;
    }
    gather4_rows((uint32_t)__cvta_generic_to_shared(stB + (size_t)pp * kTileElems + 4 * h * 256), map, r[0], r[1], r[2],
                 r[3], mbar);
  }
}

}  // namespace umma

// TPC row tiles of 128 rows per CTA share each K step's D blocks (the B
// operand): with TPC = 2 a step moves 3 NP tiles for two tiles' work instead
// of 2 NP for one, in 3 stages (2 with NP = 3, so that two CTAs still fit an
// SM), one accumulator per tile (no double buffer; two CTAs per SM overlap
// one's epilogue with the other's MMAs) and 512 pairs of metadata; TPC = 1
// keeps 4 stages and two accumulators.  DEEP = 1 (with TPC = 2) runs one
// CTA per SM instead: 5 stages (6 with NP = 2) to cover the copies' latency
// and two accumulators per tile (all 512 tensor-memory columns), so the
// epilogue of one run overlaps the next run's MMAs within the CTA.
template <int NP, int TPC, int DEEP = 0>
struct Q2Shape {
  static constexpr int kS = DEEP ? (NP == 2 ? 6 : 5) : TPC == 2 ? (NP == 2 ? 3 : 2) : umma::kStages;   // stages
  static constexpr int kMP = TPC == 2 ? 512 : umma::kMetaPairs;    // pairs per CTA segment
  static constexpr int kNB = TPC == 2 && !DEEP ? 1 : 2;            // accumulator buffers
  static constexpr int kCols = kNB * TPC * 128;                    // tensor-memory columns
};

template <int NP, int TPC, int DEEP>
__global__ void __launch_bounds__(192) k_q2_umma(DevPlan P, MixPlan X, const int* list, const long long* slot0,
                                                 int n_slots, int a0, int a1, int FC8, int MC, int NSEG,
                                                 long long zblk, int flush, const __grid_constant__ DRows drows,
                                                 int* err) {
  // Warp roles: warp 0 lane 0 produces (bulk async copies into a stage
  // ring, completion counted in bytes on full[s]); warp 1 lane 0 issues the
  // MMAs (all piece products of a pair into the TMEM accumulators, commits
  // free the stage / hand the accumulators to the epilogue); warps 2..5 read
  // the accumulators (each its 32-lane quarter of tensor memory) and dot
  // them with grad C_AF.  No block barrier inside the pipeline.
  using namespace umma;
  constexpr int KS = Q2Shape<NP, TPC, DEEP>::kS, KMP = Q2Shape<NP, TPC, DEEP>::kMP, NB = Q2Shape<NP, TPC, DEEP>::kNB;
  constexpr int TCOLS = Q2Shape<NP, TPC, DEEP>::kCols;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint16_t* stA = reinterpret_cast<uint16_t*>(smem_raw);                  // [KS][TPC][NP][kTileElems]
  uint16_t* stB = stA + (size_t)KS * TPC * NP * kTileElems;               // [KS][NP][kTileElems]
  int* m_dblk = reinterpret_cast<int*>(stB + (size_t)KS * NP * kTileElems);   // [KMP][8]
  __shared__ __align__(8) uint64_t bar_full[KS], bar_empty[KS], bar_accf[2], bar_acce[2];
  __shared__ uint32_t tmem_base;
  __shared__ double sg[8][3];
  __shared__ int m_q[kMetaPairs];
  __shared__ int s_nsteps;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int rem = blockIdx.x;
  const int seg = rem % NSEG;
  rem /= NSEG;
  const int MCP = (MC + TPC - 1) / TPC;
  const int mc = (rem % MCP) * TPC;   // first row tile of this CTA
  rem /= MCP;
  const int fc = rem % FC8;
  const int A = a0 + rem / FC8;   // home atom of this pass [a0, a1); slot0 counts from the pass's first pair
  const int sA = P.species[A];
  const int nA = P.n_ao[sA], mA = P.n_abf[sA];
  const int rows = mA * nA, nt = (rows + 127) >> 7;
  const int q0 = P.c_ptr[A], nq = P.c_ptr[A + 1] - q0;
  if (fc * 8 >= nq || mc * 128 >= rows || P.v_ptr[A] == P.v_ptr[A + 1]) return;
  const int ntile = min(TPC, nt - mc);   // row tiles of this CTA
  const long long s0 = slot0[P.v_ptr[A]];
  const long long s1 = A + 1 < a1 ? slot0[P.v_ptr[A + 1]] : (long long)n_slots;
  const long long p0 = s0 + (long long)seg * KMP;
  const int np = (int)max(0ll, min((long long)KMP, s1 - p0));
  if (np <= 0) return;
  const int row0 = mc * 128;
  int qf[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int j = fc * 8 + i;
    qf[i] = (j < nq && P.c_keep[q0 + j]) ? q0 + j : -1;
  }
  // D block (units of 256 elements) of every (pair, F), or -1, from the table
  {
    const int4* tab = reinterpret_cast<const int4*>(X.q2tab + ((long long)fc * n_slots + p0) * 8);
    for (int e = tid; e < np * 2; e += blockDim.x) reinterpret_cast<int4*>(m_dblk)[e] = tab[e];
  }
  const uint32_t mfull = (uint32_t)__cvta_generic_to_shared(&bar_full[0]);
  const uint32_t mempty = (uint32_t)__cvta_generic_to_shared(&bar_empty[0]);
  const uint32_t maccf = (uint32_t)__cvta_generic_to_shared(&bar_accf[0]);
  const uint32_t macce = (uint32_t)__cvta_generic_to_shared(&bar_acce[0]);
  if (tid < 24) sg[tid / 3][tid % 3] = 0.0;
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < KS; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mfull + 8 * s));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mempty + 8 * s));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(maccf + 8 * b));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(macce + 8 * b));
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 1) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst), "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {   // K steps: pairs with a kept D block for at least one of the 8 F, in order
    int n = 0;
    for (int t0 = 0; t0 < np; t0 += 32) {
      const int t = t0 + lane;
      bool any = false;
      if (t < np) {
        const int4 u = *reinterpret_cast<const int4*>(m_dblk + t * 8);
        const int4 v = *reinterpret_cast<const int4*>(m_dblk + t * 8 + 4);
        any = !(u.x < 0 && u.y < 0 && u.z < 0 && u.w < 0 && v.x < 0 && v.y < 0 && v.z < 0 && v.w < 0);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, any);
      if (any) m_q[n + __popc(bal & ((1u << lane) - 1u))] = t;
      n += __popc(bal);
    }
    if (lane == 0) s_nsteps = n;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t taddr = tmem_base;
  const int nsteps = s_nsteps;
  const int nruns = (nsteps + flush - 1) / flush;

  if (warp == 0 && !X.stall_q2) {
    // producer warp: every lane waits for the stage, then lanes issue the
    // copies of one stage in parallel (lane 0 also posts the byte count)
    const uint32_t abytes = (uint32_t)ntile * NP * kTileElems * 2;
    const uint32_t bytes = abytes + (uint32_t)NP * kTileElems * 2;
    for (int k = 0; k < nsteps; ++k) {
      const int s = k % KS;
      const int t = m_q[k];
      if (k >= KS && !mbar_wait<kMixTryNs>(mempty + 8 * s, (uint32_t)((k / KS - 1) & 1))) s_abort = 1;
      __syncwarp();
      if (s_abort) break;
      // lane 0: the NP Z piece tiles of the CTA's row tiles (contiguous, one
      // copy); lanes 1 .. 2 NP: the eight D blocks of each piece, four per gather
      if (lane == 0) {
        mbar_expect_tx(mfull + 8 * s, bytes);
        bulk_g2s((uint32_t)__cvta_generic_to_shared(stA + (size_t)s * TPC * NP * kTileElems),
                 X.Zst + (p0 + t) * zblk + (long long)mc * NP * kTileElems, abytes, mfull + 8 * s);
      }
      stage_d<NP>(lane, stB + (size_t)s * NP * kTileElems, m_dblk + t * 8, &drows.map, drows.zero_row, mfull + 8 * s);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: D f32, A/B bf16, both K-major, N = 128, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
      for (int r = 0; r < nruns && !s_abort; ++r) {
        const int b = r % NB;
        if (r >= NB && !mbar_wait<kMixTryNs>(macce + 8 * b, (uint32_t)((r / NB - 1) & 1))) {
          s_abort = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t dacc = taddr + 128u * TPC * b;
        const int k1 = min(nsteps, (r + 1) * flush);
        for (int k = r * flush; k < k1; ++k) {
          const int s = k % KS;
          if (!mbar_wait<kMixTryNs>(mfull + 8 * s, (uint32_t)((k / KS) & 1))) {
            s_abort = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(stA + (size_t)s * TPC * NP * kTileElems);
          const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(stB + (size_t)s * NP * kTileElems);
          const bool fs = k == r * flush;   // first step of the run: each tile's first product overwrites
          for (int j = 0; j < ntile; ++j)
#pragma unroll
            for (int sum = NP - 1; sum >= 0; --sum)
#pragma unroll
              for (int ia = 0; ia <= sum; ++ia) {
                const int ib = sum - ia;
                const uint64_t ad = sdesc(a0 + (j * NP + ia) * kTileElems * 2);
                const uint64_t bd = sdesc(b0 + ib * kTileElems * 2);
                const uint32_t acc = (fs && sum == NP - 1 && ia == 0) ? 0u : 1u;
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dacc + 128u * j),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
              }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mempty + 8 * s)
                       : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(maccf + 8 * b)
                     : "memory");
      }
    }
  } else {
    // epilogue: warps 2..5, tensor-memory lane quarter q = warp % 4
    const int q = warp & 3;
    double gd[8][3];
#pragma unroll
    for (int i = 0; i < 8; ++i) gd[i][0] = gd[i][1] = gd[i][2] = 0.0;
    for (int run = 0; run < nruns; ++run) {
      const int b = run % NB;
      if (!mbar_wait<kMixTryNs>(maccf + 8 * b, (uint32_t)((run / NB) & 1))) {
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      for (int j = 0; j < ntile; ++j) {
      const int r = row0 + 128 * j + q * 32 + lane;
      const bool rv = r < rows;
#pragma unroll
      for (int c0 = 0; c0 < 128; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(taddr + ((uint32_t)(q * 32) << 16) + 128u * (TPC * b + j) + c0, v);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = (c0 >> 4) + h;
          if (!rv || qf[i] < 0) continue;
          // grad C_AF rows in gc_off order: the warp's 32 rows of one 4-column
          // group are 512 consecutive bytes; columns f >= n_ao(F) are zero on
          // both sides
          const float4* dC4 = reinterpret_cast<const float4*>(X.Cm + X.cm_off[qf[i]] + (long long)NP * nt * 2048) +
                              (r >> 7) * 512 + (r & 127);
          float4 w[3][4];
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int f4 = 0; f4 < 4; ++f4) w[c][f4] = dC4[c * nt * 512 + f4 * 128];
          float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
          for (int f4 = 0; f4 < 4; ++f4) {
            const float x0 = __uint_as_float(v[h * 16 + 4 * f4]), x1 = __uint_as_float(v[h * 16 + 4 * f4 + 1]);
            const float x2 = __uint_as_float(v[h * 16 + 4 * f4 + 2]), x3 = __uint_as_float(v[h * 16 + 4 * f4 + 3]);
            g0 = fmaf(w[0][f4].x, x0, fmaf(w[0][f4].y, x1, fmaf(w[0][f4].z, x2, fmaf(w[0][f4].w, x3, g0))));
            g1 = fmaf(w[1][f4].x, x0, fmaf(w[1][f4].y, x1, fmaf(w[1][f4].z, x2, fmaf(w[1][f4].w, x3, g1))));
            g2 = fmaf(w[2][f4].x, x0, fmaf(w[2][f4].y, x1, fmaf(w[2][f4].z, x2, fmaf(w[2][f4].w, x3, g2))));
          }
          gd[i][0] += (double)g0;
          gd[i][1] += (double)g1;
          gd[i][2] += (double)g2;
        }
      }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(macce + 8 * b) : "memory");
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double w = warp_sum_d(gd[i][c]);
        if (lane == 0 && w != 0.0) {
          if (P.fxC) dev::add_gC(P, 3 * qf[i] + c, -2.0 * w);   // deterministic plan: straight into the exact cell
          else atomicAdd(&sg[i][c], w);
        }
      }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(TCOLS));
  if (tid < 24) {
    const int i = tid / 3, c = tid % 3;
    if (qf[i] >= 0 && sg[i][c] != 0.0) dev::add_gC(P, 3 * qf[i] + c, -2.0 * sg[i][c]);
  }
  if (tid == 0 && s_abort) atomicExch(err, 1);
}

// ------------------------------------------------------------ tcgen05 Y build
// Y^{XZ}[(alpha,x)][z] = sum_W sum_w C_XW[(alpha,x)][w] D_WZ[w][z] for a
// group of up to 8 needed keys Z of one home atom X and 128 rows: K runs over
// the kept C pairs (X,W) (one k16 step each); the B operand of key i is the
// mirror block D_ZW = D_WZ^T (rows z, columns w).  Same warp roles as
// k_q2_umma; one accumulation run; the epilogue splits the FP32 result into
// bf16 pieces and writes the Y store ([alpha][z][16], x padding zeroed).
// TPC row tiles of 128 rows per CTA share each K step's D blocks (one
// accumulator of 128 columns per tile).
// stages of the Y build's ring: 4, or 2 for two six-product tiles (so that
// two CTAs still fit an SM)
__host__ __device__ constexpr int yb_stages(int np, int tpc) { return tpc == 2 && np == 3 ? 2 : umma::kStages; }

template <int NP, int TPC>
__global__ void __launch_bounds__(192) k_ybuild_umma(DevPlan P, MixPlan X, const int* ylist, const int* gX,
                                                     const int* gS, const int* gN, int MC,
                                                     const __grid_constant__ DRows drows, int* err) {
  using namespace umma;
  constexpr int kStages = yb_stages(NP, TPC);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint16_t* stA = reinterpret_cast<uint16_t*>(smem_raw);                     // [kStages][TPC][NP][kTileElems]
  uint16_t* stB = stA + (size_t)kStages * TPC * NP * kTileElems;           // [kStages][NP][kTileElems]
  int* m_d = reinterpret_cast<int*>(stB + (size_t)kStages * NP * kTileElems);   // [kMaxCPerAtom][8]
  __shared__ int m_q[kMaxCPerAtom];
  __shared__ int s_nsteps;
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages], bar_accf;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int MCP = (MC + TPC - 1) / TPC;
  const int g = blockIdx.x / MCP, mc = (blockIdx.x - g * MCP) * TPC;   // first row tile of this CTA
  const int Xa = gX[g], kstart = gS[g], nk = gN[g];
  const int sX = P.species[Xa];
  const int mX = P.n_abf[sX], nX = P.n_ao[sX];
  const int rows = mX * nX;
  if (mc * 128 >= rows) return;
  const int ntile = min(TPC, ((rows + 127) >> 7) - mc);
  const int q0 = P.c_ptr[Xa], nq = P.c_ptr[Xa + 1] - q0;
  int ykey[8], zat[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    ykey[i] = i < nk ? ylist[kstart + i] : -1;
    zat[i] = ykey[i] >= 0 ? P.y_j[ykey[i]] : 0;
  }
  // D block of every (C pair, key), or -1, from the table
  {
    const int4* tab = reinterpret_cast<const int4*>(X.ytab + (long long)g * X.ytab_stride);
    for (int e = tid; e < nq * 2; e += blockDim.x) reinterpret_cast<int4*>(m_d)[e] = tab[e];
  }
  const uint32_t mfull = (uint32_t)__cvta_generic_to_shared(&bar_full[0]);
  const uint32_t mempty = (uint32_t)__cvta_generic_to_shared(&bar_empty[0]);
  const uint32_t maccf = (uint32_t)__cvta_generic_to_shared(&bar_accf);
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mfull + 8 * s));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mempty + 8 * s));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(maccf));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 1) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst), "r"(128 * TPC));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  __syncthreads();
  if (warp == 0) {   // K steps: kept C pairs with at least one D block among the keys, in order
    int n = 0;
    for (int t0 = 0; t0 < nq; t0 += 32) {
      const int t = t0 + lane;
      bool any = false;
      if (t < nq) {
        const int4 u = *reinterpret_cast<const int4*>(m_d + t * 8);
        const int4 v = *reinterpret_cast<const int4*>(m_d + t * 8 + 4);
        any = !(u.x < 0 && u.y < 0 && u.z < 0 && u.w < 0 && v.x < 0 && v.y < 0 && v.z < 0 && v.w < 0);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, any);
      if (any) m_q[n + __popc(bal & ((1u << lane) - 1u))] = t;
      n += __popc(bal);
    }
    if (lane == 0) s_nsteps = n;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t taddr = tmem_base;
  const int nsteps = s_nsteps;

  if (warp == 0) {
    const uint32_t abytes = (uint32_t)ntile * NP * kTileElems * 2;
    const uint32_t bytes = abytes + (uint32_t)NP * kTileElems * 2;
    for (int k = 0; k < nsteps; ++k) {
      const int s = k % kStages;
      if (k >= kStages && !mbar_wait<kMixTryNs>(mempty + 8 * s, (uint32_t)((k / kStages - 1) & 1))) s_abort = 1;
      __syncwarp();
      if (s_abort) break;
      const int t = m_q[k];
      // lane 0: the NP C piece tiles of the CTA's row tiles (contiguous, one
      // copy); lanes 1 .. 2 NP: the eight mirror D blocks of each piece, four per gather
      if (lane == 0) {
        mbar_expect_tx(mfull + 8 * s, bytes);
        bulk_g2s((uint32_t)__cvta_generic_to_shared(stA + (size_t)s * TPC * NP * kTileElems),
                 X.Cm + X.cm_off[q0 + t] + (long long)mc * NP * kTileElems, abytes, mfull + 8 * s);
      }
      stage_d<NP>(lane, stB + (size_t)s * NP * kTileElems, m_d + t * 8, &drows.map, drows.zero_row, mfull + 8 * s);
    }
  } else if (warp == 1) {
    if (lane == 0 && nsteps > 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
      for (int k = 0; k < nsteps; ++k) {
        const int s = k % kStages;
        if (!mbar_wait<kMixTryNs>(mfull + 8 * s, (uint32_t)((k / kStages) & 1))) {
          s_abort = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(stA + (size_t)s * TPC * NP * kTileElems);
        const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(stB + (size_t)s * NP * kTileElems);
        for (int j = 0; j < ntile; ++j)
#pragma unroll
          for (int sum = NP - 1; sum >= 0; --sum)
#pragma unroll
            for (int ia = 0; ia <= sum; ++ia) {
              const uint64_t ad = sdesc(a0 + (j * NP + ia) * kTileElems * 2);
              const uint64_t bd = sdesc(b0 + (sum - ia) * kTileElems * 2);
              const uint32_t acc = (k == 0 && sum == NP - 1 && ia == 0) ? 0u : 1u;
              asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                           " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr + 128u * j),
                           "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mempty + 8 * s)
                     : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(maccf)
                   : "memory");
    }
  } else {
    // epilogue (warps 2..5): the accumulator (rows (alpha, x), columns
    // (key, z)) passes through shared memory, two keys at a time, in the
    // stage ring (idle once the last MMA has completed), so that the Y store
    // and its FP32 copy are written as whole 16-byte chunks of complete
    // (alpha, z) rows, x padding included.  An alpha whose rows straddle two
    // row tiles is written element by element by both; the tile that holds
    // x = n_ao - 1 writes its padding.
    const int q = warp & 3;
    const int et = tid - 64;
    float* ep = reinterpret_cast<float*>(smem_raw);   // [128][33]
    bool have = nsteps > 0;
    if (have) {
      if (!mbar_wait<kMixTryNs>(maccf, 0u)) {
        s_abort = 1;
        have = false;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    for (int jt = 0; jt < ntile; ++jt) {
    const int row0 = (mc + jt) * 128;
    const int rend = min(row0 + 128, rows);
    const int alF = (row0 + nX - 1) / nX, alL = rend / nX - 1;
    const int nal = max(0, alL - alF + 1);
    const int alA = row0 / nX, alB = (rend - 1) / nX;
    for (int c0 = 0; c0 < 128; c0 += 32) {
      {
        uint32_t v[32];
        if (have) {
          tmem_ld32(taddr + ((uint32_t)(q * 32) << 16) + 128u * jt + c0, v);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0u;
        }
        float* er = ep + (q * 32 + lane) * 33;
#pragma unroll
        for (int j = 0; j < 32; ++j) er[j] = __uint_as_float(v[j]);
      }
      asm volatile("bar.sync 1, 128;\n" ::: "memory");
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int i = (c0 >> 4) + h;
        if (ykey[i] < 0) continue;
        const int nZ = P.n_ao[P.species[zat[i]]];
        uint16_t* Yo = X.Ysp + P.y_off[ykey[i]];
        float* Yf = X.Yf ? X.Yf + P.y_off[ykey[i]] / NP : nullptr;
        const bool cm = X.ycm != 0;   // Ysp rows alpha (64), K = (z, x) in core-matrix order
        const int KZc = 16 * nZ;
        const long long plane = cm ? 64LL * KZc : (long long)mX * nZ * 16;
        const float* eh = ep + h * 16;
        // bf16 pieces: chunk (alpha, z, half) holds x = 8 half .. 8 half + 7
        // (core-matrix order: consecutive threads take consecutive alpha, whose
        // chunks are 16 bytes apart)
        for (int c = et; c < nal * nZ * 2; c += 128) {
          int hf, al, zz;
          if (cm) {
            const int r2 = c / nal;
            al = alF + (c - r2 * nal);
            hf = r2 & 1;
            zz = r2 >> 1;
          } else {
            const int az = c >> 1;
            hf = c & 1;
            al = alF + az / nZ;
            zz = az - (az / nZ) * nZ;
          }
          const int rl = al * nX - row0 + 8 * hf;
          float f0[4], f1[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            f0[k] = 8 * hf + k < nX ? eh[(rl + k) * 33 + zz] : 0.f;
            f1[k] = 8 * hf + 4 + k < nX ? eh[(rl + 4 + k) * 33 + zz] : 0.f;
          }
          uint2 p0[NP], p1[NP];
          split4<NP>(f0, p0);
          split4<NP>(f1, p1);
          uint16_t* yo = Yo + (cm ? cmx(al, zz * 16 + 8 * hf, KZc) : ((long long)al * nZ + zz) * 16 + 8 * hf);
#pragma unroll
          for (int pp = 0; pp < NP; ++pp)
            *reinterpret_cast<uint4*>(yo + pp * plane) = make_uint4(p0[pp].x, p0[pp].y, p1[pp].x, p1[pp].y);
        }
        // FP32 copy as [z][alpha][16]; chunk c (16 bytes) of row alpha holds
        // x = 4 (c ^ sw) .. + 3 with sw = 2 ((alpha >> 1) & 1), so that four
        // consecutive rows read two adjacent chunks each from distinct
        // shared-memory banks
        if (Yf) {
          for (int c = et; c < nal * nZ * 4; c += 128) {
            const int cq = c & 3, za = c >> 2, zz = za / nal, al = alF + (za - zz * nal);
            const int x0 = 4 * (cq ^ (2 * ((al >> 1) & 1)));
            const int rl = al * nX - row0 + x0;
            float4 o;
            o.x = x0 < nX ? eh[rl * 33 + zz] : 0.f;
            o.y = x0 + 1 < nX ? eh[(rl + 1) * 33 + zz] : 0.f;
            o.z = x0 + 2 < nX ? eh[(rl + 2) * 33 + zz] : 0.f;
            o.w = x0 + 3 < nX ? eh[(rl + 3) * 33 + zz] : 0.f;
            *reinterpret_cast<float4*>(Yf + ((long long)zz * mX + al) * 16 + 4 * cq) = o;
          }
        }
        // transposed pieces for the second product: accumulator row (alpha, x)
        // with the 16 z of key i (z >= n_ao(Z) zero); every row of the tile
        // is this CTA's own
        if (X.YspT) {
          // row-major tiles [(alpha, x)][16 z], or (ycm) rows alpha (64), K = (x, z) in core-matrix order
          uint16_t* ytb = X.YspT + X.y_idx[ykey[i]] * X.yT_blk;
          uint16_t* yt = ytb + (long long)row0 * 16;
          const long long tplane = cm ? 64LL * 16 * nX : X.yT_blk / NP;
          // (core-matrix order: consecutive threads take consecutive alpha of one
          // (x, half), whose chunks are 16 bytes apart; rows outside the tile skipped)
          const int nala = alB - alA + 1;
          const int nct = cm ? nala * nX * 2 : (rend - row0) * 2;
          for (int c = et; c < nct; c += 128) {
            int rl, hz;
            if (cm) {
              const int r2 = c / nala, al = alA + (c - r2 * nala), x = r2 >> 1;
              hz = r2 & 1;
              rl = al * nX + x - row0;
              if (rl < 0 || row0 + rl >= rend) continue;
            } else {
              rl = c >> 1;
              hz = c & 1;
            }
            float f0[4], f1[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              f0[k] = 8 * hz + k < nZ ? eh[rl * 33 + 8 * hz + k] : 0.f;
              f1[k] = 8 * hz + 4 + k < nZ ? eh[rl * 33 + 8 * hz + 4 + k] : 0.f;
            }
            uint2 p0[NP], p1[NP];
            split4<NP>(f0, p0);
            split4<NP>(f1, p1);
            uint16_t* dst = yt + rl * 16 + 8 * hz;
            if (cm) {
              const int r = row0 + rl, al = r / nX, x = r - al * nX;
              dst = ytb + cmx(al, x * 16 + 8 * hz, 16 * nX);
            }
#pragma unroll
            for (int pp = 0; pp < NP; ++pp)
              *reinterpret_cast<uint4*>(dst + pp * tplane) = make_uint4(p0[pp].x, p0[pp].y, p1[pp].x, p1[pp].y);
          }
        }
        // alphas shared with a neighbouring row tile
#pragma unroll 1
        for (int pa = 0; pa < 2; ++pa) {
          const int al = pa ? alB : alA;
          if (pa ? (alB <= alL || alB == alA) : (alA >= alF)) continue;
          const int r0 = max(row0, al * nX), nr = min(rend, (al + 1) * nX) - r0;
          for (int c = et; c < nr * nZ; c += 128) {
            const int zz = c / nr, r = r0 + (c - zz * nr), x = r - al * nX;
            const float y = eh[(r - row0) * 33 + zz];
            uint16_t pc[NP];
            split_f<NP>(y, pc);
            const long long o = cm ? cmx(al, zz * 16, KZc) : ((long long)al * nZ + zz) * 16;   // + x (x < 16)
            const int sw = 2 * ((al >> 1) & 1);
            float* yr = Yf ? Yf + ((long long)zz * mX + al) * 16 : nullptr;
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) Yo[pp * plane + o + (cm ? ((x >> 3) << 6) + (x & 7) : x)] = pc[pp];
            if (yr) yr[(((x >> 2) ^ sw) << 2) + (x & 3)] = y;
            if (x == nX - 1)
              for (int xp = nX; xp < 16; ++xp) {
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) Yo[pp * plane + o + (cm ? ((xp >> 3) << 6) + (xp & 7) : xp)] = 0;
                if (yr) yr[(((xp >> 2) ^ sw) << 2) + (xp & 3)] = 0.f;
              }
          }
        }
      }
      asm volatile("bar.sync 1, 128;\n" ::: "memory");
    }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(128 * TPC));
  if (tid == 0 && s_abort) atomicExch(err, 1);
}

// Groups of up to 8 consecutive needed keys of one home atom (the needed keys
// of atom X sit at positions [y_idx[y_ptr[X]], y_idx[y_ptr[X+1]]) of the list).
__global__ void k_ygroups(DevPlan P, const long long* y_idx, const long long* y_total, int* gcnt, const long long* goff,
                          int* gX, int* gS, int* gN, int phase) {
  for (int Xa = blockIdx.x * blockDim.x + threadIdx.x; Xa < P.N; Xa += gridDim.x * blockDim.x) {
    const long long first = P.y_ptr[Xa] < P.nY ? y_idx[P.y_ptr[Xa]] : *y_total;
    const long long last = Xa + 1 < P.N && P.y_ptr[Xa + 1] < P.nY ? y_idx[P.y_ptr[Xa + 1]] : *y_total;
    const int n = (int)(last - first);
    if (phase == 0) {
      gcnt[Xa] = (n + 7) / 8;
    } else {
      const long long o = goff[Xa];
      for (int g = 0; g * 8 < n; ++g) {
        gX[o + g] = Xa;
        gS[o + g] = (int)(first + 8 * g);
        gN[o + g] = min(8, n - 8 * g);
      }
    }
  }
}

// D block (256-element units) of every (key group g, C slot t of its home
// atom X, key i) of the Y build, or -1 (C pair dropped, key absent, D block
// screened out); the Y build's flops are counted here.
__global__ void k_ytab(DevPlan P, MixPlan X, const int* ylist, const int* gX, const int* gS, const int* gN,
                       int ngroups) {
  const int TC = X.ytab_stride >> 3;
  const long long total = (long long)ngroups * X.ytab_stride;
  double fl = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e & 7);
    const long long gt = e >> 3;
    const int g = (int)(gt / TC), t = (int)(gt - (long long)g * TC);
    const int Xa = gX[g];
    const int q0 = P.c_ptr[Xa], nq = P.c_ptr[Xa + 1] - q0;
    if (t >= nq) continue;
    const int key = i < gN[g] ? ylist[gS[g] + i] : -1;
    int md = -1;
    if (key >= 0 && P.c_keep[q0 + t]) {
      const int* Rz = P.y_R + 3 * key;
      const int* Rw = P.c_R + 3 * (q0 + t);
      const int w = P.c_j[q0 + t], z = P.y_j[key];
      const int di = dlut_get(P, w, z, Rz[0] - Rw[0], Rz[1] - Rw[1], Rz[2] - Rw[2]);
      if (di >= 0 && P.Dkept[di] != 0.0) {
        const int mi = dlut_get(P, z, w, Rw[0] - Rz[0], Rw[1] - Rz[1], Rw[2] - Rz[2]);
        md = (int)(X.dsp_off[mi] >> 8);
        const int sX = P.species[Xa];
        fl += 2.0 * P.n_abf[sX] * P.n_ao[sX] * P.n_ao[P.species[z]] * P.n_ao[P.species[w]];
      }
    }
    X.ytab[e] = md;
  }
  fl = warp_sum_d(fl);
  if ((threadIdx.x & 31) == 0 && fl != 0.0) atomicAdd(&P.acc[ACC_FY], fl);
}

// D block of every (group fc of 8 C slots of the pair's home atom A, pair
// slot of the second product, i), or -1; the Q2 product's flops are counted
// here.
__global__ void k_q2tab(DevPlan P, MixPlan X, const int* list, int n_slots, int FC8) {
  const long long total = (long long)n_slots * FC8 * 8;
  double fl = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e & 7);
    const long long r = e >> 3;
    const int fc = (int)(r / n_slots), slot = (int)(r - (long long)fc * n_slots);
    const int p = list[slot];
    const int A = P.v_home[p];
    const int q0 = P.c_ptr[A], nq = P.c_ptr[A + 1] - q0;
    const int j = fc * 8 + i;
    int db = -1;
    if (j < nq && P.c_keep[q0 + j]) {
      const int qf = q0 + j, b = P.v_j[p];
      const int* Rb = P.v_R + 3 * p;
      const int* Rf = P.c_R + 3 * qf;
      const int d = dlut_get(P, P.c_j[qf], b, Rb[0] - Rf[0], Rb[1] - Rf[1], Rb[2] - Rf[2]);
      if (d >= 0 && P.Dkept[d] != 0.0) {
        db = (int)(X.dsp_off[d] >> 8);
        const int sA = P.species[A];
        fl += 2.0 * P.n_abf[sA] * P.n_ao[sA] * P.n_ao[P.species[b]] * P.n_ao[P.species[P.c_j[qf]]];
      }
    }
    X.q2tab[e] = db;
  }
  fl = warp_sum_d(fl);
  if ((threadIdx.x & 31) == 0 && fl != 0.0) atomicAdd(&P.acc[ACC_F2], fl);
}

size_t ybuild_umma_smem(int np, int tpc) {
  return (size_t)(tpc + 1) * yb_stages(np, tpc) * np * umma::kTileElems * sizeof(uint16_t) +
         (size_t)kMaxCPerAtom * 8 * sizeof(int);
}

size_t q2_umma_smem(int np, int tpc) {
  if (tpc >= 2) {   // 3: two tiles, the deep pipeline
    const int ks = tpc == 3 ? (np == 2 ? Q2Shape<2, 2, 1>::kS : Q2Shape<3, 2, 1>::kS)
                            : (np == 2 ? Q2Shape<2, 2>::kS : Q2Shape<3, 2>::kS);
    return (size_t)ks * 3 * np * umma::kTileElems * sizeof(uint16_t) + (size_t)Q2Shape<2, 2>::kMP * 8 * sizeof(int);
  }
  return (size_t)2 * Q2Shape<2, 1>::kS * np * umma::kTileElems * sizeof(uint16_t) +
         (size_t)Q2Shape<2, 1>::kMP * 8 * sizeof(int);
}

int grid_for(long long n, int cap) {
  long long g = n < 1 ? 1 : n;
  return (int)(g > cap ? cap : g);
}

}  // namespace

long long mixed_launch_count() { return g_mix_launches; }

long long ytab_size(int ngroups, int maxC) { return (long long)ngroups * 8 * maxC; }
long long q2tab_size(int n_slots, int FC) { return (long long)n_slots * ((FC * 4 + 7) / 8) * 8; }

int q2_umma_segments(int max_pairs_per_atom, int np, int tpc) {
  const int kmp = tpc >= 2 ? Q2Shape<2, 2>::kMP : Q2Shape<2, 1>::kMP;
  return (max_pairs_per_atom + kmp - 1) / kmp;
}

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

cudaError_t launch_ygroups(const DevPlan& P, const long long* y_idx, const long long* y_total, int* gcnt,
                           const long long* goff, int* gX, int* gS, int* gN, int phase, cudaStream_t s) {
  ++g_mix_launches;
  k_ygroups<<<(P.N + 255) / 256, 256, 0, s>>>(P, y_idx, y_total, gcnt, goff, gX, gS, gN, phase);
  return cudaGetLastError();
}

cudaError_t launch_ybuild_mma(const DevPlan& P, const MixPlan& X, int np, const int* ylist, const int* gX,
                              const int* gS, const int* gN, int ngroups, int MC, const DRows& drows, int* err,
                              cudaStream_t s) {
  if (ngroups == 0) return cudaSuccess;
  g_mix_launches += 2;
  k_ytab<<<grid_for(((long long)ngroups * X.ytab_stride + 255) / 256, 152 * 16), 256, 0, s>>>(P, X, ylist, gX, gS, gN,
                                                                                          ngroups);
  const int tpc = X.ybtpc == 1 ? 1 : 2;
  const long long grid = (long long)ngroups * ((MC + tpc - 1) / tpc);
  const size_t sm = ybuild_umma_smem(np, tpc);
  if (np == 2 && tpc == 2) k_ybuild_umma<2, 2><<<(unsigned)grid, 192, sm, s>>>(P, X, ylist, gX, gS, gN, MC, drows, err);
  else if (np == 2) k_ybuild_umma<2, 1><<<(unsigned)grid, 192, sm, s>>>(P, X, ylist, gX, gS, gN, MC, drows, err);
  else if (tpc == 2) k_ybuild_umma<3, 2><<<(unsigned)grid, 192, sm, s>>>(P, X, ylist, gX, gS, gN, MC, drows, err);
  else k_ybuild_umma<3, 1><<<(unsigned)grid, 192, sm, s>>>(P, X, ylist, gX, gS, gN, MC, drows, err);
  return cudaGetLastError();
}

cudaError_t launch_t1_lists(const DevPlan& P, const MixPlan& X, int phase, cudaStream_t s) {
  ++g_mix_launches;
  if (P.nC > 0) k_t1_lists<<<grid_for((P.nC + 7) / 8, 152 * 16), 256, 0, s>>>(P, X, phase);
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

cudaError_t set_mixed_smem_limits(int np) {
  const void* f[7] = {
      np == 2 ? (const void*)k_ybuild_umma<2, 2> : (const void*)k_ybuild_umma<3, 2>,
      np == 2 ? (const void*)k_ybuild_umma<2, 1> : (const void*)k_ybuild_umma<3, 1>,
      np == 2 ? (const void*)k_q2_umma<2, 2, 0> : (const void*)k_q2_umma<3, 2, 0>,
      np == 2 ? (const void*)k_q2_umma<2, 2, 1> : (const void*)k_q2_umma<3, 2, 1>,
      np == 2 ? (const void*)k_q2_umma<2, 1, 0> : (const void*)k_q2_umma<3, 1, 0>,
      np == 2 ? (const void*)k_term1_mma<2> : (const void*)k_term1_mma<3>,
      np == 2 ? (const void*)k_term2_pairs<2> : (const void*)k_term2_pairs<3>};
  for (const void* k : f) {
    const cudaError_t e = allow_max_dynamic_smem(k);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
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
                             int n, int a0, int a1, int MAmax, int KZmax, long long zblk, int zrows, int FC, int MC,
                             int nseg, int flush, const DRows& drows, size_t smem, int* err, cudaStream_t s,
                             bool pairs_done) {
  if (n == 0 || a1 <= a0) return cudaSuccess;
  g_mix_launches += pairs_done ? 2 : 3;
  const int FC8 = (FC * 4 + 7) / 8;     // groups of 8 C slots for the tcgen05 kernel
  k_q2tab<<<grid_for(((long long)n * FC8 * 8 + 255) / 256, 152 * 16), 256, 0, s>>>(P, X, list, n, FC8);
  const int tpc = X.q2tpc == 1 ? 1 : 2, deep = X.q2tpc == 3 ? 1 : 0;   // row tiles per CTA; the deep pipeline
  const size_t sq = q2_umma_smem(np, X.q2tpc == 1 ? 1 : (deep ? 3 : 2));
  const long long grid = (long long)(a1 - a0) * FC8 * ((MC + tpc - 1) / tpc) * nseg;
  auto q2 = [&](auto kern) {
    kern<<<(unsigned)grid, 192, sq, s>>>(P, X, list, slot0, n, a0, a1, FC8, MC, nseg, zblk, flush, drows, err);
  };
  if (np == 2) {
    if (!pairs_done)
      k_term2_pairs<2><<<grid_for(n, 152 * 32), kWarps * 32, smem, s>>>(P, X, list, n, MAmax, KZmax, zblk, zrows);
    if (tpc == 1) q2(k_q2_umma<2, 1, 0>);
    else if (deep) q2(k_q2_umma<2, 2, 1>);
    else q2(k_q2_umma<2, 2, 0>);
  } else {
    if (!pairs_done)
      k_term2_pairs<3><<<grid_for(n, 152 * 32), kWarps * 32, smem, s>>>(P, X, list, n, MAmax, KZmax, zblk, zrows);
    if (tpc == 1) q2(k_q2_umma<3, 1, 0>);
    else if (deep) q2(k_q2_umma<3, 2, 1>);
    else q2(k_q2_umma<3, 2, 0>);
  }
  return cudaGetLastError();
}

}  // namespace hfx
