// Split-precision kernels for block shapes beyond the tensor-memory kernels'
// tiles: n_ao up to 32 per species (the perovskite Cs blocks, n_ao 18) and
// n_abf up to 128.
//
// Same factorisation and the same bf16 piece products as hfx_mixed.cu (NP
// pieces per operand, the products (i, j) with i + j < NP, FP32 accumulation
// in warp-level MMAs, FP64 screening, gradients and reductions), organised
// like the FP64 kernels of hfx_kernels.cu so that any n_ao and n_abf fit.
// Operands are split into bf16 pieces once, into stores that the kernels copy
// from:
//   D pieces   per D block, NP planes [rup16(n_ao(I))][rup16(n_ao(J))]   (plan)
//   C pieces   per C pair, NP planes [alpha][rup8(n_ao(A) n_ao(F))]        (per call)
//   Y pieces   per needed key (X; Z), NP planes [alpha][z][rup16(n_ao(X))] (Y build)
//   Z pieces   per second-product pair, NP planes [(alpha, a)][KZ]        (per pass)
// V and grad V stay FP64 (one pair per CTA reads them once).
//
//   k_ybuild_w  Y^{XZ}[alpha][x][z] = sum_W sum_w C_XW[alpha][x][w] D_WZ[w][z]
//               per group of up to 8 keys (X; Z) of one home atom X and 64 rows
//               (alpha, x), over the kept C pairs (X, W)
//   k_term1_w   per kept (A,B) of the first exchange product, over its kept F
//               and ranges of a:
//                 U[beta][(a,f)] = sum_b D_AB[a][b] Y^{BF}[beta][b][f]
//                 R += C_AF . U^T   (E, g^V after every few F)
//                 Q  = V_AB . U     (dotted with grad C_AF at once)
//   k_term2_w   per kept (A,B) of the second product, over ranges of a:
//                 R2 += Y^{AB} . Y^{BA}   (K = (a, b))
//                 Z   = V_AB . Y^{BA}     (rows (alpha, a), to the Z pieces)
//   k_q2_w      per (A, 128 rows (alpha, a), 8 C pairs (A,F)):
//                 Q2 = sum_B Z^{AB} . D_FB^T, dotted with grad C_AF
// (Eq. exx_expand by the distributive law; Eq. Fexx1 for the gradients.)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "hfx_accum.cuh"
#include "hfx_device.cuh"

namespace hfx {
namespace {

using namespace dev;

constexpr int kWThreads = 256;   // 8 warps per CTA
constexpr int kWarpsW = kWThreads / 32;
constexpr int kFlushF = 8;       // F per FP32 run of R in the first product
std::atomic<long long> g_wide_launches{0};

__device__ __forceinline__ int rup8(int x) { return (x + 7) & ~7; }

// 16-byte asynchronous copies global -> shared (both 16-byte aligned)
__device__ __forceinline__ void cpa16(void* sdst, const void* gsrc) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// piece pp of (x0, x1) packed as one 32-bit word, x0 in the low half
template <int NP>
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t (&w)[NP]) {
  uint16_t p0[NP], p1[NP];
  split_f<NP>(x0, p0);
  split_f<NP>(x1, p1);
#pragma unroll
  for (int pp = 0; pp < NP; ++pp) w[pp] = pack2(p0[pp], p1[pp]);
}

// element e of a [rows][S] bf16 plane set (NP planes of `plane` elements): the NP pieces of x
template <int NP>
__device__ __forceinline__ void put_pieces(uint16_t* base, long long plane, int e, float x) {
  uint16_t pc[NP];
  split_f<NP>(x, pc);
#pragma unroll
  for (int pp = 0; pp < NP; ++pp) base[pp * plane + e] = pc[pp];
}

template <int NV, int NW = kWarpsW>
__device__ void block_sum_w(double (&v)[NV], double* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum_d(v[i]);
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i * NW + w] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = 0.0;
    for (int k = 0; k < NW; ++k) t += red[i * NW + k];
    v[i] = t;
  }
  __syncthreads();
}

// Warps per CTA of the two product kernels (one CTA per SM, bound by shared
// memory) and the R tile pairs each warp keeps: NW * RP >= 64 pairs covers
// n_abf <= 128.
constexpr int kPW = 16;
constexpr int kPRP = 64 / kPW;

// R (M = alpha tiles, N = beta tiles) as pairs of beta tiles; pair k of warp w
// is pair index w + 8 k of the MT x ceil(NT / 2) pairs.
struct RTiles {
  int MT, NTP, NT;
  __device__ RTiles(int MA, int MB) : MT(MA >> 4), NTP(((MB >> 3) + 1) >> 1), NT(MB >> 3) {}
  __device__ int count() const { return MT * NTP; }
};

// acc += A . B^T over K in [0, K): A rows (M) at As (stride SA), B rows (N) at Bs
// (stride SB), both K-contiguous, for tile pair (mt, nt0, nt0 + 1).
template <int NP>
__device__ __forceinline__ void gemm_pair_kk(float (&acc)[2][4], const uint16_t* As, long long pa, int SA,
                                             const uint16_t* Bs, long long pb, int SB, int mt, int nt0, bool two, int K) {
  const int lane = threadIdx.x & 31;
  const int nt1 = two ? nt0 + 1 : nt0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t af[NP][4], b0[NP][2], b1[NP][2];
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
      ldm_x4(af[pp], As + pp * pa + (long long)(mt * 16 + (lane & 15)) * SA + k0 + ((lane >> 4) << 3));
      ldm_x2(b0[pp], Bs + pp * pb + (long long)(nt0 * 8 + (lane & 7)) * SB + k0 + (((lane >> 3) & 1) << 3));
      ldm_x2(b1[pp], Bs + pp * pb + (long long)(nt1 * 8 + (lane & 7)) * SB + k0 + (((lane >> 3) & 1) << 3));
    }
    mma_split2<NP>(acc[0], af, b0, acc[1], af, b1);
  }
}

// acc += A . B over K in [0, K): A rows (M) K-contiguous at As (stride SA), B
// rows (K) N-contiguous at Bs (stride SB), for tile pair (mt, nt0, nt0 + 1).
template <int NP>
__device__ __forceinline__ void gemm_pair_kn(float (&acc)[2][4], const uint16_t* As, long long pa, int SA,
                                             const uint16_t* Bs, long long pb, int SB, int mt, int nt0, bool two, int K) {
  const int lane = threadIdx.x & 31;
  const int nt1 = two ? nt0 + 1 : nt0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t af[NP][4], b0[NP][2], b1[NP][2];
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) {
      ldm_x4(af[pp], As + pp * pa + (long long)(mt * 16 + (lane & 15)) * SA + k0 + ((lane >> 4) << 3));
      ldm_x2_trans(b0[pp], Bs + pp * pb + (long long)(k0 + (lane & 15)) * SB + nt0 * 8);
      ldm_x2_trans(b1[pp], Bs + pp * pb + (long long)(k0 + (lane & 15)) * SB + nt1 * 8);
    }
    mma_split2<NP>(acc[0], af, b0, acc[1], af, b1);
  }
}

// ------------------------------------------------------------------ D pieces
// D block k (fixed for the plan) -> NP bf16 planes of rup16(n_ao(I)) x
// rup16(n_ao(J)), row-major, zero padded, at Dw + dw_off[k].
template <int NP>
__global__ void k_dsplit_w(DevPlan P, uint16_t* Dw, const long long* dw_off) {
  for (long long k = blockIdx.x; k < P.n_d; k += gridDim.x) {
    const int I = P.Didx[5 * k], J = P.Didx[5 * k + 1];
    const int na = P.n_ao[P.species[I]], nb = P.n_ao[P.species[J]];
    const int pa = rup16(na), pb = rup16(nb);
    const double* src = P.Dval + P.Doff[k];
    uint16_t* out = Dw + dw_off[k];
    for (int e = threadIdx.x; e < pa * pb; e += blockDim.x) {
      const int a = e / pb, b = e - a * pb;
      put_pieces<NP>(out, (long long)pa * pb, e, (a < na && b < nb) ? (float)src[a * nb + b] : 0.f);
    }
  }
}

// ------------------------------------------------------------------ C pieces
// Kept C pair q (evaluated this call, FP64) -> at Cw + cw_off[q]: NP bf16
// planes of [alpha][rup8(n_ao(A) n_ao(F))] (columns (a, f) as in the FP64
// block, zero padded; the first product's layout), then NP planes of
// [(alpha, a)][rup16(n_ao(F))] (the Y build's A operand: every row starts on
// a 16-byte boundary).
__host__ __device__ inline int cw_cols(int nA, int nF) { return (nA * nF + 7) & ~7; }

// ... and grad C in FP32 (dCf, the layout of P.dCst), which the first
// product's Q epilogue reads in MMA-fragment order: half the bytes of the
// FP64 blocks, and the same values (the epilogue rounds to FP32 anyway).
template <int NP>
__global__ void k_cpieces_w(DevPlan P, uint16_t* Cw, const long long* cw_off, float* dCf) {
  for (int q = blockIdx.x; q < P.nC; q += gridDim.x) {
    if (!P.c_keep[q]) continue;
    const int sA = P.species[P.c_home[q]], sF = P.species[P.c_j[q]];
    const int mA = P.n_abf[sA], nA = P.n_ao[sA], nF = P.n_ao[sF];
    const int naf = nA * nF, CW = cw_cols(nA, nF), KW = rup16(nF);
    const double* src = P.Cst + P.c_off[q];
    uint16_t* out = Cw + cw_off[q];
    for (int e = threadIdx.x; e < mA * CW; e += blockDim.x) {
      const int al = e / CW, c = e - al * CW;
      put_pieces<NP>(out, (long long)mA * CW, e, c < naf ? (float)src[(long long)al * naf + c] : 0.f);
    }
    uint16_t* cy = out + (long long)NP * mA * CW;
    for (int e = threadIdx.x; e < mA * nA * KW; e += blockDim.x) {
      const int r = e / KW, c = e - r * KW;
      put_pieces<NP>(cy, (long long)mA * nA * KW, e, c < nF ? (float)src[(long long)r * nF + c] : 0.f);
    }
    const double* dsrc = P.dCst + 3 * P.c_off[q];
    float* dst = dCf + 3 * P.c_off[q];
    for (int e = threadIdx.x; e < 3 * mA * naf; e += blockDim.x) dst[e] = (float)dsrc[e];
  }
}

// ------------------------------------------------------------------ Y build
// CTA = (key group g, 64-row block rb).  Warp w: rows 16 (w & 3) of the block,
// keys 4 (w >> 2) .. + 3 of the group, all z of each key (n_ao(Z) <= 32: four
// column tiles).  K steps: 16 columns w of one kept C pair (X, W) with a D
// block among the keys, two steps in flight (16-byte asynchronous copies):
//   As[2][NP][64][24]          C_XW rows (alpha, x), columns w (the padded C pieces)
//   Bs[2][NP][16][8 * 32 + 8]  D_{W Z_i} rows w, columns (i, z) (the D pieces)
constexpr int kYRows = 64;
constexpr int kYSA = 24;
constexpr int kYSB = 8 * 32 + 8;
size_t ybuild_w_smem(int np) { return (size_t)2 * np * (kYRows * kYSA + 16 * kYSB) * sizeof(uint16_t); }

template <int NP>
__global__ void __launch_bounds__(kWThreads) k_ybuild_w(DevPlan P, uint16_t* __restrict__ Yp,
                                                        const uint16_t* __restrict__ Cw, const long long* cw_off,
                                                        const uint16_t* __restrict__ Dw, const long long* dw_off,
                                                        const int* ylist, const int* gX, const int* gS, const int* gN,
                                                        int RB) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr long long pA = kYRows * kYSA, pB = 16 * kYSB;
  uint16_t* As0 = reinterpret_cast<uint16_t*>(smem);   // [2][NP][64][kYSA]
  uint16_t* Bs0 = As0 + 2 * NP * pA;                   // [2][NP][16][kYSB]
  __shared__ int m_dw[kMaxCPerAtom][8];   // D piece block of (C pair t, key i) in 256-element units, or -1
  __shared__ int m_step[2 * kMaxCPerAtom];
  __shared__ int s_key[8], s_zat[8], s_nz[8];
  __shared__ int s_nsteps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int g = blockIdx.x / RB, rb = blockIdx.x - g * RB;
  const int Xa = gX[g], kstart = gS[g], nk = gN[g];
  const int sX = P.species[Xa];
  const int mX = P.n_abf[sX], nX = P.n_ao[sX], KX = rup16(nX);
  const int rows = mX * nX;
  const int row0 = rb * kYRows;
  if (row0 >= rows) return;
  const int q0 = P.c_ptr[Xa], nq = P.c_ptr[Xa + 1] - q0;
  if (threadIdx.x < 8) {
    const int i = threadIdx.x;
    const int key = i < nk ? ylist[kstart + i] : -1;
    s_key[i] = key;
    s_zat[i] = key >= 0 ? P.y_j[key] : 0;
    s_nz[i] = key >= 0 ? P.n_ao[P.species[P.y_j[key]]] : 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nq * 8; e += blockDim.x) {
    const int t = e >> 3, i = e & 7;
    const int q = q0 + t;
    int dw = -1;
    if (s_key[i] >= 0 && P.c_keep[q]) {
      const int* Rw = P.c_R + 3 * q;
      const int* Rz = P.y_R + 3 * s_key[i];
      const int di = dlut_get(P, P.c_j[q], s_zat[i], Rz[0] - Rw[0], Rz[1] - Rw[1], Rz[2] - Rw[2]);
      if (di >= 0 && P.Dkept[di] != 0.0) dw = (int)(dw_off[di] >> 8);
    }
    m_dw[t][i] = dw;
  }
  __syncthreads();
  if (threadIdx.x == 0) {   // K steps: (kept C pair with a D block among the keys, 16-column step)
    int n = 0;
    double fl = 0.0;
    for (int t = 0; t < nq; ++t) {
      bool any = false;
      const int nW = P.n_ao[P.species[P.c_j[q0 + t]]];
      for (int i = 0; i < 8; ++i)
        if (m_dw[t][i] >= 0) {
          any = true;
          fl += 2.0 * rows * s_nz[i] * nW;
        }
      if (!any) continue;
      for (int k0 = 0; k0 < nW; k0 += 16) m_step[n++] = (t << 8) | k0;
    }
    s_nsteps = n;
    if (rb == 0) atomicAdd(&P.acc[ACC_FY], fl);
  }
  __syncthreads();
  const int nsteps = s_nsteps;
  const int mt = warp & 3, kh = warp >> 2;
  int nz4[4];   // n_ao(Z) of this warp's four keys
#pragma unroll
  for (int ii = 0; ii < 4; ++ii) nz4[ii] = s_nz[4 * kh + ii];
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
  // copies of step k into buffer k & 1 (rows past the block and columns past
  // the keys' D blocks are not copied: they only meet discarded results)
  auto issue = [&](int k) {
    const int t = m_step[k] >> 8, k0 = m_step[k] & 255;
    const int q = q0 + t;
    const int nW = P.n_ao[P.species[P.c_j[q]]], pw = rup16(nW);
    const uint16_t* Cy = Cw + cw_off[q] + (long long)NP * mX * cw_cols(nX, nW);   // [(alpha, x)][pw]
    const long long cplane = (long long)rows * pw;
    uint16_t* As = As0 + (k & 1) * NP * pA;
    uint16_t* Bs = Bs0 + (k & 1) * NP * pB;
    const int nr = min(kYRows, rows - row0);
    for (int e = threadIdx.x; e < NP * nr * 2; e += blockDim.x) {
      const int pp = e / (nr * 2), rr = e - pp * nr * 2, r = rr >> 1, h = rr & 1;
      cpa16(As + pp * pA + r * kYSA + 8 * h, Cy + pp * cplane + (long long)(row0 + r) * pw + k0 + 8 * h);
    }
    for (int i = 0; i < 8; ++i) {
      const int dw = m_dw[t][i];
      if (dw < 0) continue;
      const int pz = rup16(s_nz[i]), ch = pz >> 3;
      const uint16_t* Dg = Dw + ((long long)dw << 8) + (long long)k0 * pz;   // rows w of D_{W Z_i} pieces [pw][pz]
      const long long dplane = (long long)pw * pz;
      for (int e = threadIdx.x; e < NP * 16 * ch; e += blockDim.x) {
        const int pp = e / (16 * ch), rr = e - pp * 16 * ch, w = rr / ch, c = rr - w * ch;
        cpa16(Bs + pp * pB + w * kYSB + i * 32 + 8 * c, Dg + pp * dplane + (long long)w * pz + 8 * c);
      }
    }
  };
  if (nsteps > 0) issue(0);
  cpa_commit();
  for (int k = 0; k < nsteps; ++k) {
    if (k + 1 < nsteps) issue(k + 1);
    cpa_commit();
    cpa_wait<1>();
    __syncthreads();   // step k's operands are in shared memory
    const int t = m_step[k] >> 8;
    const uint16_t* As = As0 + (k & 1) * NP * pA;
    const uint16_t* Bs = Bs0 + (k & 1) * NP * pB;
    uint32_t af[NP][4];
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) ldm_x4(af[pp], As + pp * pA + (mt * 16 + (lane & 15)) * kYSA + ((lane >> 4) << 3));
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      const int i = 4 * kh + ii;
      if (m_dw[t][i] < 0) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        if (nt * 8 >= nz4[ii]) break;
        uint32_t bf[NP][2];
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) ldm_x2_trans(bf[pp], Bs + pp * pB + (lane & 15) * kYSB + i * 32 + nt * 8);
        mma_split<NP>(acc[ii][nt], af, bf);
      }
    }
    __syncthreads();   // buffer k & 1 is free for step k + 2
  }
  cpa_wait<0>();
  // Y pieces [alpha][z][x] (x padded to rup16(n_ao(X)) with zeros, written
  // with the row x = n_ao(X) - 1)
#pragma unroll
  for (int ii = 0; ii < 4; ++ii) {
    const int key = s_key[4 * kh + ii];
    if (key < 0) continue;
    const int nZ = nz4[ii];
    uint16_t* Y = Yp + P.y_off[key];
    const long long plane = (long long)mX * nZ * KX;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      if (nt * 8 >= nZ) break;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int row = row0 + mt * 16 + gid + ((c & 2) ? 8 : 0);
        const int z = nt * 8 + 2 * tig + (c & 1);
        if (row < rows && z < nZ) {
          const int al = row / nX, x = row - al * nX;
          const long long o = ((long long)al * nZ + z) * KX;
          put_pieces<NP>(Y, plane, (int)(o + x), acc[ii][nt][c]);
          if (x == nX - 1)
            for (int xp = nX; xp < KX; ++xp)
#pragma unroll
              for (int pp = 0; pp < NP; ++pp) Y[pp * plane + o + xp] = 0;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ term 1
// Shared memory (bf16 planes; strides are multiples of 8 elements with an
// odd count of 16-byte chunks, so that ldmatrix rows hit distinct banks):
//   Vs[NP][MA][MB + 8]   V_AB (rows alpha, columns beta; zero padded)
//   Ds[NP][48][40]       D_AB (rows a, columns b; zero padded; 16 rows from any a0 < 32)
//   Cs[NP][MA][KC + 8]   C_AF columns (a, f) of the current range of a
//   Us[NP][MB][KC + 8]   U of the same columns (rows beta)
struct T1W {
  int MA, MB, KC, da;
};

__host__ __device__ inline size_t term1w_smem(int np, int MA, int MB, int KC) {
  return (size_t)np * 2 * ((size_t)MA * (MB + 8) + 48 * 40 + (size_t)MA * (KC + 8) + (size_t)MB * (KC + 8));
}

template <int NP>
__global__ void __launch_bounds__(kPW * 32, 1) k_term1_w(DevPlan P, const uint16_t* __restrict__ Yp,
                                                       const uint16_t* __restrict__ Cw, const long long* cw_off,
                                                       const uint16_t* __restrict__ Dw, const long long* dw_off,
                                                       const float* __restrict__ dCf, const int* list, int n_list,
                                                       T1W S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[4 * kPW];
  __shared__ double s_g[3];
  __shared__ int s_q;   // C pair whose grad C partials are in s_g
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int MA = S.MA, MB = S.MB;
  const int SV = MB + 8, SD = 40, SK = S.KC + 8;
  const long long pV = (long long)MA * SV, pD = 48 * SD, pC = (long long)MA * SK, pU = (long long)MB * SK;
  uint16_t* Vs = reinterpret_cast<uint16_t*>(smem);
  uint16_t* Ds = Vs + NP * pV;
  uint16_t* Cs = Ds + NP * pD;
  uint16_t* Us = Cs + NP * pC;
  for (int kk = blockIdx.x; kk < n_list; kk += gridDim.x) {
    const int p = list[kk];
    const int A = P.v_home[p], b = P.v_j[p];
    const int* Rb = P.v_R + 3 * p;
    const int sA = P.species[A], sB = P.species[b];
    const int nA = P.n_ao[sA], nB = P.n_ao[sB], mA = P.n_abf[sA], mB = P.n_abf[sB];
    const int MAp = rup16(mA), MBp = rup16(mB), KB = rup16(nB);
    const double* V = P.Vst + P.v_off[p];
    const int nvb = mA * mB;
    const int pa = rup16(nA);
    const uint16_t* Dg = Dw + dw_off[P.v_didx[p]];   // D_AB pieces [pa][KB]
    __syncthreads();   // previous pair done with every buffer
    if (threadIdx.x == 0) {
      s_g[0] = s_g[1] = s_g[2] = 0.0;
      s_q = -1;
    }
    for (int e = threadIdx.x; e < MA * SV; e += blockDim.x) {
      const int al = e / SV, be = e - al * SV;
      put_pieces<NP>(Vs, pV, e, (al < mA && be < mB) ? (float)V[al * mB + be] : 0.f);
    }
    for (int e = threadIdx.x; e < 48 * SD; e += blockDim.x) {
      const int a = e / SD, bb = e - a * SD;
      const bool in = a < pa && bb < KB;
#pragma unroll
      for (int pp = 0; pp < NP; ++pp) Ds[pp * pD + e] = in ? Dg[(long long)pp * pa * KB + a * KB + bb] : (uint16_t)0;
    }
    // U rows beyond n_abf(B) stay zero (they meet the zero V columns in Q)
    for (int e = threadIdx.x; e < (MB - mB) * SK; e += blockDim.x)
#pragma unroll
      for (int pp = 0; pp < NP; ++pp) Us[pp * pU + (long long)mB * SK + e] = 0;
    const RTiles rt(MAp, MBp);
    float racc[kPRP][2][4];
#pragma unroll
    for (int i = 0; i < kPRP; ++i)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int c = 0; c < 4; ++c) racc[i][h][c] = 0.f;
    double ev[4] = {0.0, 0.0, 0.0, 0.0};
    // E and g^V of the R run so far (FP32 dot, FP64 sum), then R restarts
    auto flush_r = [&]() {
      float evf[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < kPRP; ++i) {
        const int pr = warp + kPW * i;
        if (pr >= rt.count()) break;
        const int mt = pr / rt.NTP, nt0 = 2 * (pr - mt * rt.NTP);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int al = mt * 16 + gid + ((c & 2) ? 8 : 0);
            const int be = (nt0 + h) * 8 + 2 * tig + (c & 1);
            if (al < mA && be < mB) {
              const int o = al * mB + be;
              const float r = racc[i][h][c];
              evf[0] = fmaf((float)V[o], r, evf[0]);
              evf[1] = fmaf((float)V[nvb + o], r, evf[1]);
              evf[2] = fmaf((float)V[2 * nvb + o], r, evf[2]);
              evf[3] = fmaf((float)V[3 * nvb + o], r, evf[3]);
            }
            racc[i][h][c] = 0.f;
          }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) ev[c] += (double)evf[c];
    };
    const int q0 = P.c_ptr[A];
    double fl = 0.0;
    int nf = 0;
    for (int wd = 0; wd < kMaskWords; ++wd) {
      unsigned bits = P.v_mask[(size_t)p * kMaskWords + wd];
      while (bits) {
        const int s = __ffs(bits) - 1;
        bits &= bits - 1u;
        const int q = q0 + wd * 32 + s;
        const int f = P.c_j[q];
        const int* Rf = P.c_R + 3 * q;
        const int nF = P.n_ao[P.species[f]];
        const int yc = ylut_get(P, b, f, Rf[0] - Rb[0], Rf[1] - Rb[1], Rf[2] - Rb[2]);
        const uint16_t* Y = Yp + P.y_off[yc];          // NP planes [beta][f][KB] (b padded)
        const long long yplane = (long long)mB * nF * KB;
        const int CW = cw_cols(nA, nF);
        const uint16_t* C = Cw + cw_off[q];             // NP planes [alpha][(a, f)] (row length CW)
        const long long cplane = (long long)mA * CW;
        const float* dC = dCf + 3 * P.c_off[q];   // grad C_AF in FP32 (k_cpieces_w)
        const long long nc = (long long)mA * nA * nF;
        const int rowsU = mB * nF;
        float gq[3] = {0.f, 0.f, 0.f};
        for (int a0 = 0; a0 < nA; a0 += S.da) {
          const int dA = min(S.da, nA - a0);
          const int dcols = dA * nF, KCc = rup16(dcols);
          __syncthreads();   // the previous range's products are done with Cs and Us
          if (threadIdx.x == 0 && s_q >= 0 && s_q != q) {   // grad C partials of the previous F
            dev::add_gC(P, 3 * s_q + 0, -2.0 * s_g[0]);
            dev::add_gC(P, 3 * s_q + 1, -2.0 * s_g[1]);
            dev::add_gC(P, 3 * s_q + 2, -2.0 * s_g[2]);
            s_g[0] = s_g[1] = s_g[2] = 0.0;
          }
          if (threadIdx.x == 0) s_q = q;
          // C_AF columns (a, f), a in [a0, a0 + dA): contiguous in each row alpha
          // of the C pieces; 16-byte copies where the range starts on a
          // 16-byte boundary (a range of 8 a: it ends on one too, or at the
          // row's zero padding), else element copies
          const int c0 = a0 * nF;
          if ((c0 & 7) == 0 && ((dcols & 7) == 0 || a0 + dA == nA)) {
            const int nch = (dcols + 7) >> 3;
            for (int e = threadIdx.x; e < NP * mA * nch; e += blockDim.x) {
              const int pp = e / (mA * nch), rr = e - pp * mA * nch, al = rr / nch, c = rr - al * nch;
              cpa16(Cs + pp * pC + al * SK + 8 * c, C + pp * cplane + (long long)al * CW + c0 + 8 * c);
            }
            const int cz = nch * 8;
            for (int e = threadIdx.x; e < mA * (KCc - cz); e += blockDim.x) {
              const int al = e / (KCc - cz), c = cz + (e - al * (KCc - cz));
#pragma unroll
              for (int pp = 0; pp < NP; ++pp) Cs[pp * pC + al * SK + c] = 0;
            }
            cpa_commit();
          } else {
            for (int e = threadIdx.x; e < mA * KCc; e += blockDim.x) {
              const int al = e / KCc, c = e - al * KCc;
#pragma unroll
              for (int pp = 0; pp < NP; ++pp)
                Cs[pp * pC + al * SK + c] = c < dcols ? C[pp * cplane + (long long)al * CW + c0 + c] : (uint16_t)0;
            }
          }
          // U columns past the range stay zero up to the 16-column step
          for (int e = threadIdx.x; e < mB * (KCc - dcols); e += blockDim.x) {
            const int be = e / (KCc - dcols), c = dcols + (e - be * (KCc - dcols));
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) Us[pp * pU + (long long)be * SK + c] = 0;
          }
          // U^T[a][(beta, f)] = sum_b D_AB[a][b] Y^{BF}[beta][b][f]: rows a0 .. a0 + 15 of D_AB
          // (the A fragments, kept for the range), columns (beta, f) eight at a
          // time from the Y pieces (rows (beta, f), K = b); rows a >= a0 + dA unused
          {
            uint32_t af[2][NP][4];
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
#pragma unroll
              for (int pp = 0; pp < NP; ++pp)
                ldm_x4(af[ks][pp], Ds + pp * pD + (a0 + (lane & 15)) * SD + ks * 16 + ((lane >> 4) << 3));
            for (int nt = warp; nt * 8 < rowsU; nt += kPW) {
              float acc[4] = {0.f, 0.f, 0.f, 0.f};
              const int rn = nt * 8 + gid;
              const bool in = rn < rowsU;
#pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                if (ks * 16 >= KB) break;
                uint32_t bf[NP][2];
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) {
                  const uint16_t* yr = Y + pp * yplane + (long long)rn * KB + ks * 16 + 2 * tig;
                  bf[pp][0] = in ? *reinterpret_cast<const uint32_t*>(yr) : 0u;
                  bf[pp][1] = in ? *reinterpret_cast<const uint32_t*>(yr + 8) : 0u;
                }
                mma_split<NP>(acc, af[ks], bf);
              }
              // acc[0], acc[1]: row a0 + gid, columns (beta, f) = nt * 8 + 2 tig, + 1
              if (gid < dA) {
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                  const int r = nt * 8 + 2 * tig + c;
                  if (r < rowsU) {
                    const int be = r / nF, ff = r - be * nF;
                    put_pieces<NP>(Us, pU, be * SK + gid * nF + ff, acc[c]);
                  }
                }
              }
            }
          }
          cpa_wait<0>();
          __syncthreads();   // Cs and Us complete
          // R += C_AF . U^T (M = alpha, N = beta, K = this range's columns)
#pragma unroll
          for (int i = 0; i < kPRP; ++i) {
            const int pr = warp + kPW * i;
            if (pr >= rt.count()) break;
            const int mt = pr / rt.NTP, nt0 = 2 * (pr - mt * rt.NTP);
            gemm_pair_kk<NP>(racc[i], Cs, pC, SK, Us, pU, SK, mt, nt0, nt0 + 1 < rt.NT, KCc);
          }
          // Q = V_AB . U (M = alpha, N = columns, K = beta), dotted with grad C_AF
          {
            const int NTQ = rup8(dcols) >> 3, NPQ = (NTQ + 1) >> 1;
            const int npairs = (MAp >> 4) * NPQ;
            for (int pr = warp; pr < npairs; pr += kPW) {
              const int mt = pr / NPQ, nt0 = 2 * (pr - mt * NPQ);
              float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
              gemm_pair_kn<NP>(acc, Vs, pV, SV, Us, pU, SK, mt, nt0, nt0 + 1 < NTQ, MBp);
#pragma unroll
              for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  const int al = mt * 16 + gid + ((c & 2) ? 8 : 0);
                  const int n = (nt0 + h) * 8 + 2 * tig + (c & 1);
                  if (al < mA && n < dcols && nt0 + h < NTQ) {
                    const long long ci = (long long)al * nA * nF + a0 * nF + n;
                    const float v = acc[h][c];
                    gq[0] = fmaf((float)dC[ci], v, gq[0]);
                    gq[1] = fmaf((float)dC[nc + ci], v, gq[1]);
                    gq[2] = fmaf((float)dC[2 * nc + ci], v, gq[2]);
                  }
                }
            }
          }
        }
        // this F's grad C partials into the shared FP64 sums (flushed at the next F or at the end)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float w = warp_sum_f(gq[c]);
          if (lane == 0) {
            if (P.fxC) dev::add_gC(P, 3 * q + c, -2.0 * (double)w);   // deterministic plan: straight into the exact cell
            else atomicAdd(&s_g[c], (double)w);
          }
        }
        fl += 2.0 * mB * nA * nB * nF + 4.0 * mA * mB * nA * nF;
        if (++nf % kFlushF == 0) flush_r();
      }
    }
    flush_r();
    block_sum_w<4, kPW>(ev, red);   // also orders the s_g additions before the flush below
    if (threadIdx.x == 0) {
      if (s_q >= 0) {
        dev::add_gC(P, 3 * s_q + 0, -2.0 * s_g[0]);
        dev::add_gC(P, 3 * s_q + 1, -2.0 * s_g[1]);
        dev::add_gC(P, 3 * s_q + 2, -2.0 * s_g[2]);
      }
      dev::add_E(P, -ev[0]);
      dev::add_gV(P, 3 * p + 0, -ev[1]);
      dev::add_gV(P, 3 * p + 1, -ev[2]);
      dev::add_gV(P, 3 * p + 2, -ev[3]);
      atomicAdd(&P.acc[ACC_F1], fl);
    }
  }
}

// ------------------------------------------------------------------ term 2
// k_term2_w, one CTA per kept (A,B) pair (slot s of the pass's list); shared
// memory (bf16 planes):
//   Vs[NP][MA][MB + 8]   V_AB
//   Ya[NP][MA][KC + 8]   Y^{AB} columns (a, b), a in the current range
//   Yb[NP][MB][KC + 8]   Y^{BA} as [beta][(a, b)], same columns
// R2 gives E and g^V; Z = V_AB . Y^{BA} goes to the Z store of slot s as NP
// bf16 planes of rows (alpha, a), columns b (row stride KZ, columns
// n_ao(B) .. rup16(n_ao(B)) - 1 zero), for k_q2_w.
struct T2W {
  int MA, MB, KC, da, KZ;
  long long zplane;    // elements per piece plane of a slot (most rows x KZ)
};

__host__ __device__ inline size_t term2w_smem(int np, int MA, int MB, int KC) {
  return (size_t)np * 2 * ((size_t)MA * (MB + 8) + (size_t)MA * (KC + 8) + (size_t)MB * (KC + 8));
}

template <int NP>
__global__ void __launch_bounds__(kPW * 32, 1) k_term2_w(DevPlan P, const uint16_t* __restrict__ Yp,
                                                       uint16_t* __restrict__ Zw, const int* list, int n_list, T2W S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[4 * kPW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int MA = S.MA, MB = S.MB;
  const int SV = MB + 8, SK = S.KC + 8;
  const long long pV = (long long)MA * SV, pA = (long long)MA * SK, pB = (long long)MB * SK;
  uint16_t* Vs = reinterpret_cast<uint16_t*>(smem);
  uint16_t* Ya = Vs + NP * pV;
  uint16_t* Yb = Ya + NP * pA;
  for (int kk = blockIdx.x; kk < n_list; kk += gridDim.x) {
    const int p = list[kk];
    const int A = P.v_home[p], b = P.v_j[p];
    const int* Rb = P.v_R + 3 * p;
    const int sA = P.species[A], sB = P.species[b];
    const int nA = P.n_ao[sA], nB = P.n_ao[sB], mA = P.n_abf[sA], mB = P.n_abf[sB];
    const int MAp = rup16(mA), MBp = rup16(mB);
    const int y1 = ylut_get(P, A, b, Rb[0], Rb[1], Rb[2]);
    const int y2 = ylut_get(P, b, A, -Rb[0], -Rb[1], -Rb[2]);
    const int KA = rup16(nA), KB = rup16(nB);
    const uint16_t* Yab = Yp + P.y_off[y1];   // Y^{AB} pieces [alpha][b][a] (a padded to KA)
    const uint16_t* Yba = Yp + P.y_off[y2];   // Y^{BA} pieces [beta][a][b] (b padded to KB)
    const long long plA = (long long)mA * nB * KA, plB = (long long)mB * nA * KB;
    const double* V = P.Vst + P.v_off[p];
    const int nvb = mA * mB;
    uint16_t* Z = Zw + (long long)kk * NP * S.zplane;   // NP planes [(alpha, a)][KZ]
    __syncthreads();   // previous pair done with every buffer
    {   // zero columns n_ao(B) .. rup16(n_ao(B)) - 1 (K padding of k_q2_w)
      const int pad = rup16(nB) - nB;
      for (int e = threadIdx.x; e < mA * nA * pad; e += blockDim.x) {
        const int r = e / pad, c = nB + (e - r * pad);
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) Z[pp * S.zplane + (long long)r * S.KZ + c] = 0;
      }
    }
    for (int e = threadIdx.x; e < MA * SV; e += blockDim.x) {
      const int al = e / SV, be = e - al * SV;
      put_pieces<NP>(Vs, pV, e, (al < mA && be < mB) ? (float)V[al * mB + be] : 0.f);
    }
    // Y^{BA} rows beyond n_abf(B) stay zero (K of Z)
    for (int e = threadIdx.x; e < (MB - mB) * SK; e += blockDim.x)
#pragma unroll
      for (int pp = 0; pp < NP; ++pp) Yb[pp * pB + (long long)mB * SK + e] = 0;
    const RTiles rt(MAp, MBp);
    float racc[kPRP][2][4];
#pragma unroll
    for (int i = 0; i < kPRP; ++i)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int c = 0; c < 4; ++c) racc[i][h][c] = 0.f;
    for (int a0 = 0; a0 < nA; a0 += S.da) {
      const int dA = min(S.da, nA - a0);
      const int dcols = dA * nB, KCc = rup16(dcols);
      __syncthreads();   // the previous range is done with Ya and Yb
      // columns c = (b, a - a0): Y^{AB} rows (alpha, b) hold a contiguously,
      // Y^{BA} rows (beta, a) hold b contiguously; both are read as 16-byte
      // vectors (a0 and the row lengths are multiples of 8)
      for (int e = threadIdx.x; e < mA * KCc; e += blockDim.x) {   // padding columns
        const int al = e / KCc, c = e - al * KCc;
        if (c >= dcols)
#pragma unroll
          for (int pp = 0; pp < NP; ++pp) Ya[pp * pA + al * SK + c] = 0;
      }
      for (int e = threadIdx.x; e < mB * KCc; e += blockDim.x) {
        const int be = e / KCc, c = e - be * KCc;
        if (c >= dcols)
#pragma unroll
          for (int pp = 0; pp < NP; ++pp) Yb[pp * pB + be * SK + c] = 0;
      }
      for (int e = threadIdx.x; e < NP * mA * nB; e += blockDim.x) {   // Y^{AB}: the dA a of a row
        const int pp = e / (mA * nB), r = e - pp * mA * nB, al = r / nB, bb = r - al * nB;
        const uint16_t* src = Yab + pp * plA + ((long long)al * nB + bb) * KA + a0;
        uint16_t* d = Ya + pp * pA + al * SK + bb * dA;
        if ((a0 & 7) == 0) {   // a0 + 8 <= rup8(n_ao(A)) <= the row length: one 16-byte vector
          const uint4 v = *reinterpret_cast<const uint4*>(src);
          const uint16_t* h = reinterpret_cast<const uint16_t*>(&v);
          for (int j = 0; j < dA; ++j) d[j] = h[j];
        } else {
          for (int j = 0; j < dA; ++j) d[j] = src[j];
        }
      }
      const int nbc = (nB + 7) >> 3;
      for (int e = threadIdx.x; e < NP * mB * dA * nbc; e += blockDim.x) {   // Y^{BA}: 8 b at once
        const int pp = e / (mB * dA * nbc), r = e - pp * mB * dA * nbc;
        const int be = r / (dA * nbc), r2 = r - be * dA * nbc, a = r2 / nbc, bc = r2 - a * nbc;
        const uint4 v = *reinterpret_cast<const uint4*>(Yba + pp * plB + ((long long)be * nA + a0 + a) * KB + 8 * bc);
        const uint16_t* h = reinterpret_cast<const uint16_t*>(&v);
        uint16_t* d = Yb + pp * pB + be * SK + a;
        for (int j = 0; j < 8 && 8 * bc + j < nB; ++j) d[(8 * bc + j) * dA] = h[j];
      }
      __syncthreads();
      // R2 += Y^{AB} . Y^{BA} (M = alpha, N = beta, K = (a, b) of the range)
#pragma unroll
      for (int i = 0; i < kPRP; ++i) {
        const int pr = warp + kPW * i;
        if (pr >= rt.count()) break;
        const int mt = pr / rt.NTP, nt0 = 2 * (pr - mt * rt.NTP);
        gemm_pair_kk<NP>(racc[i], Ya, pA, SK, Yb, pB, SK, mt, nt0, nt0 + 1 < rt.NT, KCc);
      }
      // Z = V_AB . Y^{BA} (M = alpha, N = (a, b), K = beta) -> Z store rows (alpha, a)
      {
        const int NTZ = rup8(dcols) >> 3, NPZ = (NTZ + 1) >> 1;
        const int npairs = (MAp >> 4) * NPZ;
        for (int pr = warp; pr < npairs; pr += kPW) {
          const int mt = pr / NPZ, nt0 = 2 * (pr - mt * NPZ);
          float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
          gemm_pair_kn<NP>(acc, Vs, pV, SV, Yb, pB, SK, mt, nt0, nt0 + 1 < NTZ, MBp);
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int al = mt * 16 + gid + ((c & 2) ? 8 : 0);
              const int n = (nt0 + h) * 8 + 2 * tig + (c & 1);
              if (al < mA && n < dcols && nt0 + h < NTZ) {
                const int bb = n / dA, a = n - bb * dA;
                put_pieces<NP>(Z, S.zplane, (int)(((long long)al * nA + a0 + a) * S.KZ + bb), acc[h][c]);
              }
            }
        }
      }
    }
    // E and g^V from R2
    double ev[4] = {0.0, 0.0, 0.0, 0.0};
    {
      float evf[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < kPRP; ++i) {
        const int pr = warp + kPW * i;
        if (pr >= rt.count()) break;
        const int mt = pr / rt.NTP, nt0 = 2 * (pr - mt * rt.NTP);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int al = mt * 16 + gid + ((c & 2) ? 8 : 0);
            const int be = (nt0 + h) * 8 + 2 * tig + (c & 1);
            if (al < mA && be < mB) {
              const int o = al * mB + be;
              const float r = racc[i][h][c];
              evf[0] = fmaf((float)V[o], r, evf[0]);
              evf[1] = fmaf((float)V[nvb + o], r, evf[1]);
              evf[2] = fmaf((float)V[2 * nvb + o], r, evf[2]);
              evf[3] = fmaf((float)V[3 * nvb + o], r, evf[3]);
            }
          }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) ev[c] = (double)evf[c];
    }
    block_sum_w<4, kPW>(ev, red);
    if (threadIdx.x == 0) {
      dev::add_E(P, -ev[0]);
      dev::add_gV(P, 3 * p + 0, -ev[1]);
      dev::add_gV(P, 3 * p + 1, -ev[2]);
      dev::add_gV(P, 3 * p + 2, -ev[3]);
      atomicAdd(&P.acc[ACC_F2], 4.0 * mA * mB * nA * nB);
    }
  }
}

// k_q2_w: CTA = (home atom A of the pass, 128 rows (alpha, a), group of 8 C
// slots F of A).  Q2^{AF}[(alpha, a)][f] = sum_B sum_b Z^{AB}[(alpha, a)][b]
// D_FB[f][b] over the pairs (A,B) of the second product (one K step of
// rup16(n_ao(B)) per pair), the eight F side by side in the columns (32 per
// slot); every kQ2Run pairs the FP32 run is dotted with grad C_AF into FP64.
// Warp w: rows 16 (w & 7) .. + 15 of the block, slots 4 (w >> 3) .. + 3.
// Operands arrive by cp.async from the Z piece store and the D piece store,
// two steps in flight:
//   As[2][NP][128][KZ + 8]     Z rows, columns b
//   Bs[2][NP][8 * 32][KZ + 8]  D_FB rows (slot, f), columns b
constexpr int kQ2Threads = 512;
constexpr int kQ2Rows = 128;
constexpr int kQ2Slots = 8;
constexpr int kQ2Seg = 256;   // pairs per segment of D-block metadata
constexpr int kQ2Run = 64;    // pairs per FP32 run

__host__ __device__ inline size_t q2w_smem(int np, int KZ) {
  return (size_t)2 * np * 2 * (size_t)(kQ2Rows + kQ2Slots * 32) * (KZ + 8);
}

template <int NP>
__global__ void __launch_bounds__(kQ2Threads, 1) k_q2_w(DevPlan P, const uint16_t* __restrict__ Zw, long long zplane,
                                                        int KZ, const uint16_t* __restrict__ Dw,
                                                        const long long* __restrict__ dw_off, const int* list,
                                                        const long long* slot0, int n_slots, int a0, int a1, int RBQ,
                                                        int SG, const float* __restrict__ dCf) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int m_dw[kQ2Seg][kQ2Slots];   // D piece block of (pair, slot) in 256-element units, or -1
  __shared__ int m_step[kQ2Seg];
  __shared__ int s_nsteps;
  __shared__ int s_q[kQ2Slots], s_nf[kQ2Slots];
  __shared__ double s_ev[kQ2Threads / 32][4][3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int mt = warp & 7, sh = warp >> 3;
  const int SZ = KZ + 8;
  const long long pA = (long long)kQ2Rows * SZ, pB = (long long)kQ2Slots * 32 * SZ;
  uint16_t* As0 = reinterpret_cast<uint16_t*>(smem);
  uint16_t* Bs0 = As0 + 2 * NP * pA;
  const int per_atom = RBQ * SG;
  const int A = a0 + blockIdx.x / per_atom;
  const int rem = blockIdx.x - (A - a0) * per_atom, rb = rem / SG, sg = rem - rb * SG;
  if (A >= a1) return;
  const int sA = P.species[A], mA = P.n_abf[sA], nA = P.n_ao[sA];
  const int rows = mA * nA, row0 = rb * kQ2Rows;
  const int q0 = P.c_ptr[A], nq = P.c_ptr[A + 1] - q0;
  if (row0 >= rows || kQ2Slots * sg >= nq) return;
  if (threadIdx.x < kQ2Slots) {
    const int t = kQ2Slots * sg + threadIdx.x;
    const int q = (t < nq && P.c_keep[q0 + t]) ? q0 + t : -1;
    s_q[threadIdx.x] = q;
    s_nf[threadIdx.x] = q >= 0 ? P.n_ao[P.species[P.c_j[q]]] : 0;
  }
  for (int e = threadIdx.x; e < (kQ2Threads / 32) * 12; e += blockDim.x) (&s_ev[0][0][0])[e] = 0.0;
  __syncthreads();
  bool any = false;
#pragma unroll
  for (int i = 0; i < kQ2Slots; ++i) any = any || s_q[i] >= 0;
  if (!any) return;
  int nf4[4];
  bool live4[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    nf4[i] = s_nf[4 * sh + i];
    live4[i] = s_q[4 * sh + i] >= 0;
  }
  const long long s0 = slot0[P.v_ptr[A]];
  const long long s1 = A + 1 < a1 ? slot0[P.v_ptr[A + 1]] : (long long)n_slots;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[i][nt][c] = 0.f;
  // dot of the FP32 run with grad C_AF (FP32 products, FP64 sums per warp), then the run restarts
  auto flush = [&]() {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (!live4[i]) continue;
      const int nF = nf4[i];
      const float* dC = dCf + 3 * P.c_off[s_q[4 * sh + i]];   // grad C_AF in FP32 (k_cpieces_w)
      const long long nc = (long long)rows * nF;
      float g[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        if (nt * 8 >= nF) break;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int r = row0 + mt * 16 + gid + ((c & 2) ? 8 : 0);
          const int ff = nt * 8 + 2 * tig + (c & 1);
          if (r < rows && ff < nF) {
            const long long ci = (long long)r * nF + ff;
            const float v = acc[i][nt][c];
            g[0] = fmaf((float)dC[ci], v, g[0]);
            g[1] = fmaf((float)dC[nc + ci], v, g[1]);
            g[2] = fmaf((float)dC[2 * nc + ci], v, g[2]);
          }
          acc[i][nt][c] = 0.f;
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float w = warp_sum_f(g[c]);
        if (lane == 0) s_ev[warp][i][c] += (double)w;
      }
    }
  };
  double fl = 0.0;
  int run = 0;
  for (long long sb = s0; sb < s1; sb += kQ2Seg) {
    const int nseg = (int)min((long long)kQ2Seg, s1 - sb);
    __syncthreads();   // the previous segment is done with the metadata
    for (int e = threadIdx.x; e < nseg * kQ2Slots; e += blockDim.x) {
      const int j = e / kQ2Slots, i = e - j * kQ2Slots;
      const int q = s_q[i];
      int dw = -1;
      if (q >= 0) {
        const int pr = list[sb + j];
        const int* Rb = P.v_R + 3 * pr;
        const int* Rf = P.c_R + 3 * q;
        const int di = dlut_get(P, P.c_j[q], P.v_j[pr], Rb[0] - Rf[0], Rb[1] - Rf[1], Rb[2] - Rf[2]);
        if (di >= 0 && P.Dkept[di] != 0.0) dw = (int)(dw_off[di] >> 8);
      }
      m_dw[j][i] = dw;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int n = 0;
      for (int j = 0; j < nseg; ++j) {
        bool k = false;
#pragma unroll
        for (int i = 0; i < kQ2Slots; ++i) k = k || m_dw[j][i] >= 0;
        if (k) m_step[n++] = j;
      }
      s_nsteps = n;
    }
    __syncthreads();
    const int nsteps = s_nsteps;
    // copies of step k into buffer k & 1: Z rows of the block, D_FB of every live slot
    auto issue = [&](int k) {
      const int j = m_step[k];
      const long long slot = sb + j;
      const int nB = P.n_ao[P.species[P.v_j[list[slot]]]], KB = rup16(nB), ch = KB >> 3;
      const uint16_t* Z = Zw + slot * NP * zplane + (long long)row0 * KZ;
      uint16_t* As = As0 + (k & 1) * NP * pA;
      uint16_t* Bs = Bs0 + (k & 1) * NP * pB;
      const int zr = min(kQ2Rows, rows - row0);
      for (int e = threadIdx.x; e < NP * zr * ch; e += blockDim.x) {
        const int pp = e / (zr * ch), rr = e - pp * zr * ch, r = rr / ch, c = rr - r * ch;
        cpa16(As + pp * pA + r * SZ + 8 * c, Z + pp * zplane + (long long)r * KZ + 8 * c);
      }
      for (int i = 0; i < kQ2Slots; ++i) {
        const int dw = m_dw[j][i];
        if (dw < 0) continue;
        const int pf = rup16(s_nf[i]);
        const uint16_t* Dg = Dw + ((long long)dw << 8);
        const long long dplane = (long long)pf * KB;
        for (int e = threadIdx.x; e < NP * pf * ch; e += blockDim.x) {
          const int pp = e / (pf * ch), rr = e - pp * pf * ch, f = rr / ch, c = rr - f * ch;
          cpa16(Bs + pp * pB + (i * 32 + f) * SZ + 8 * c, Dg + pp * dplane + (long long)f * KB + 8 * c);
        }
      }
    };
    if (nsteps > 0) issue(0);
    cpa_commit();
    for (int k = 0; k < nsteps; ++k) {
      if (k + 1 < nsteps) issue(k + 1);
      cpa_commit();
      cpa_wait<1>();
      __syncthreads();   // step k's operands are in shared memory
      const int j = m_step[k];
      const int nB = P.n_ao[P.species[P.v_j[list[sb + j]]]], KB = rup16(nB);
      const uint16_t* As = As0 + (k & 1) * NP * pA;
      const uint16_t* Bs = Bs0 + (k & 1) * NP * pB;
      bool on[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) on[i] = m_dw[j][4 * sh + i] >= 0;
      for (int ks = 0; ks < KB; ks += 16) {
        uint32_t af[NP][4];
#pragma unroll
        for (int pp = 0; pp < NP; ++pp)
          ldm_x4(af[pp], As + pp * pA + (mt * 16 + (lane & 15)) * SZ + ks + ((lane >> 4) << 3));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (!on[i]) continue;
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            if (nt * 8 >= nf4[i]) break;
            uint32_t bf[NP][2];
#pragma unroll
            for (int pp = 0; pp < NP; ++pp)
              ldm_x2(bf[pp], Bs + pp * pB + ((4 * sh + i) * 32 + nt * 8 + (lane & 7)) * SZ + ks +
                                 (((lane >> 3) & 1) << 3));
            mma_split<NP>(acc[i][nt], af, bf);
          }
        }
      }
      if (rb == 0 && threadIdx.x == 0)
        for (int i = 0; i < kQ2Slots; ++i)
          if (m_dw[j][i] >= 0) fl += 2.0 * mA * nA * nB * s_nf[i];
      if (++run == kQ2Run) {
        flush();
        run = 0;
      }
      __syncthreads();   // buffer k & 1 is free for step k + 2
    }
    cpa_wait<0>();
  }
  flush();
  __syncthreads();
  if (threadIdx.x < kQ2Slots * 3) {
    const int i = threadIdx.x / 3, c = threadIdx.x - 3 * i;
    const int q = s_q[i];
    if (q >= 0) {
      double v = 0.0;
      for (int w = 0; w < 8; ++w) v += s_ev[(i >> 2) * 8 + w][i & 3][c];
      dev::add_gC(P, 3 * q + c, -2.0 * v);
    }
  }
  if (threadIdx.x == 0 && fl != 0.0) atomicAdd(&P.acc[ACC_F2], fl);
}

int grid_cap(long long n, int cap) { return (int)(n < cap ? (n > 0 ? n : 1) : cap); }

}  // namespace

long long wide_launch_count() { return g_wide_launches.load(); }

int wide_ybuild_row_blocks(int max_rows) { return (max_rows + kYRows - 1) / kYRows; }

WideShapes wide_shapes(int np, int maxABF, int maxAO, size_t limit) {
  WideShapes w{};
  w.MA = w.MB = (maxABF + 15) / 16 * 16;
  w.KZ = (maxAO + 15) / 16 * 16;
  for (int da : {8, 4, 2, 1}) {
    const int KC = (da * maxAO + 15) / 16 * 16;
    if (term1w_smem(np, w.MA, w.MB, KC) <= limit) {
      w.t1_da = da;
      w.t1_KC = KC;
      w.smem_t1 = term1w_smem(np, w.MA, w.MB, KC);
      break;
    }
  }
  for (int da : {8, 4, 2, 1}) {
    const int KC = (da * maxAO + 15) / 16 * 16;
    if (term2w_smem(np, w.MA, w.MB, KC) <= limit) {
      w.t2_da = da;
      w.t2_KC = KC;
      w.smem_t2 = term2w_smem(np, w.MA, w.MB, KC);
      break;
    }
  }
  w.smem_q2 = q2w_smem(np, w.KZ);
  // R tiles: (MA / 16) x (MB / 16) pairs over the warps, kPRP each
  w.ok = w.t1_da > 0 && w.t2_da > 0 && w.smem_q2 <= limit && (w.MA / 16) * (w.MB / 16) <= kPW * kPRP &&
         maxAO <= 32;
  return w;
}

cudaError_t set_wide_smem_limits(int np) {
  cudaError_t e = cudaSuccess;
  auto one = [&](const void* f) {
    const cudaError_t r = allow_max_dynamic_smem(f);
    if (r != cudaSuccess) e = r;
  };
  if (np == 2) {
    one((const void*)k_ybuild_w<2>);
    one((const void*)k_term1_w<2>);
    one((const void*)k_term2_w<2>);
    one((const void*)k_q2_w<2>);
  } else {
    one((const void*)k_ybuild_w<3>);
    one((const void*)k_term1_w<3>);
    one((const void*)k_term2_w<3>);
    one((const void*)k_q2_w<3>);
  }
  return e;
}

cudaError_t launch_cpieces_w(const DevPlan& P, int np, uint16_t* Cw, const long long* cw_off, float* dCf,
                             cudaStream_t s) {
  if (P.nC <= 0) return cudaSuccess;
  const int grid = grid_cap(P.nC, 1 << 16);
  if (np == 2) k_cpieces_w<2><<<grid, 256, 0, s>>>(P, Cw, cw_off, dCf);
  else k_cpieces_w<3><<<grid, 256, 0, s>>>(P, Cw, cw_off, dCf);
  ++g_wide_launches;
  return cudaGetLastError();
}

long long wide_cpieces_size(int np, int n_abf, int n_ao_a, int n_ao_f) {
  return (long long)np * n_abf * (cw_cols(n_ao_a, n_ao_f) + n_ao_a * ((n_ao_f + 15) / 16 * 16));
}

cudaError_t launch_ybuild_w(const DevPlan& P, int np, uint16_t* Yp, const uint16_t* Cw, const long long* cw_off,
                            const uint16_t* Dw, const long long* dw_off, const int* ylist, const int* gX,
                            const int* gS, const int* gN, int ngroups, int RB, cudaStream_t s) {
  if (ngroups <= 0) return cudaSuccess;
  const long long grid = (long long)ngroups * RB;
  const size_t smem = ybuild_w_smem(np);
  if (np == 2)
    k_ybuild_w<2><<<(unsigned)grid, kWThreads, smem, s>>>(P, Yp, Cw, cw_off, Dw, dw_off, ylist, gX, gS, gN, RB);
  else
    k_ybuild_w<3><<<(unsigned)grid, kWThreads, smem, s>>>(P, Yp, Cw, cw_off, Dw, dw_off, ylist, gX, gS, gN, RB);
  ++g_wide_launches;
  return cudaGetLastError();
}

cudaError_t launch_term1_w(const DevPlan& P, int np, const uint16_t* Yp, const uint16_t* Cw, const long long* cw_off,
                           const uint16_t* Dw, const long long* dw_off, const float* dCf, const int* list, int n,
                           const WideShapes& w, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const T1W S{w.MA, w.MB, w.t1_KC, w.t1_da};
  const int grid = grid_cap(n, 1 << 20);
  if (np == 2) k_term1_w<2><<<grid, kPW * 32, w.smem_t1, s>>>(P, Yp, Cw, cw_off, Dw, dw_off, dCf, list, n, S);
  else k_term1_w<3><<<grid, kPW * 32, w.smem_t1, s>>>(P, Yp, Cw, cw_off, Dw, dw_off, dCf, list, n, S);
  ++g_wide_launches;
  return cudaGetLastError();
}

long long wide_zplane(int max_rows, int KZ) { return (long long)max_rows * KZ; }

cudaError_t launch_dsplit_w(const DevPlan& P, int np, uint16_t* Dw, const long long* dw_off, cudaStream_t s) {
  if (P.n_d <= 0) return cudaSuccess;
  const int grid = grid_cap(P.n_d, 1 << 16);
  if (np == 2) k_dsplit_w<2><<<grid, 256, 0, s>>>(P, Dw, dw_off);
  else k_dsplit_w<3><<<grid, 256, 0, s>>>(P, Dw, dw_off);
  ++g_wide_launches;
  return cudaGetLastError();
}

cudaError_t launch_term2_w(const DevPlan& P, int np, const uint16_t* Yp, uint16_t* Zw, const uint16_t* Dw,
                           const long long* dw_off, const float* dCf, const int* list, const long long* slot0, int n,
                           int a0, int a1, int max_rows, int max_c, const WideShapes& w, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const T2W S{w.MA, w.MB, w.t2_KC, w.t2_da, w.KZ, wide_zplane(max_rows, w.KZ)};
  const int grid = grid_cap(n, 1 << 20);
  if (np == 2) k_term2_w<2><<<grid, kPW * 32, w.smem_t2, s>>>(P, Yp, Zw, list, n, S);
  else k_term2_w<3><<<grid, kPW * 32, w.smem_t2, s>>>(P, Yp, Zw, list, n, S);
  ++g_wide_launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int RBQ = (max_rows + kQ2Rows - 1) / kQ2Rows, SG = (max_c + kQ2Slots - 1) / kQ2Slots;
  const long long qgrid = (long long)(a1 - a0) * RBQ * SG;
  if (qgrid <= 0) return cudaSuccess;
  if (np == 2)
    k_q2_w<2><<<(unsigned)qgrid, kQ2Threads, w.smem_q2, s>>>(P, Zw, S.zplane, w.KZ, Dw, dw_off, list, slot0, n, a0, a1,
                                                             RBQ, SG, dCf);
  else
    k_q2_w<3><<<(unsigned)qgrid, kQ2Threads, w.smem_q2, s>>>(P, Zw, S.zplane, w.KZ, Dw, dw_off, list, slot0, n, a0, a1,
                                                             RBQ, SG, dCf);
  ++g_wide_launches;
  return cudaGetLastError();
}

}  // namespace hfx
