// Split-precision kernels for block shapes beyond the tensor-memory kernels'
// tiles: n_ao up to 32 per species (the perovskite Cs blocks, n_ao 18) and
// n_abf up to 128.
//
// Same factorisation and the same bf16 piece products as hfx_mixed.cu (NP
// pieces per operand, the products (i, j) with i + j < NP, FP32 accumulation
// in warp-level MMAs, FP64 screening, gradients and reductions), organised
// like the FP64 kernels of hfx_kernels.cu so that any n_ao and n_abf fit:
// operands are the FP64 blocks (C, grad C, V, grad V, D) and an FP32 store of
// the Y blocks, split into bf16 pieces where they are staged in shared memory.
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
//                 Z   = V_AB . Y^{BA}     (rows (alpha, a), shared memory)
//                 per C pair (A,F):  Q2 = Z . D_FB^T, dotted with grad C_AF
// (Eq. exx_expand by the distributive law; Eq. Fexx1 for the gradients.)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "hfx_device.cuh"

namespace hfx {
namespace {

using namespace dev;

constexpr int kWThreads = 256;   // 8 warps per CTA
constexpr int kWarpsW = kWThreads / 32;
constexpr int kRPairs = 8;       // (alpha, beta) tile pairs of R per warp (n_abf <= 128)
constexpr int kFlushF = 4;       // F per FP32 run of R in the first product
std::atomic<long long> g_wide_launches{0};

__device__ __forceinline__ int rup8(int x) { return (x + 7) & ~7; }

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

template <int NV>
__device__ void block_sum_w(double (&v)[NV], double* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum_d(v[i]);
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i * kWarpsW + w] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = 0.0;
    for (int k = 0; k < kWarpsW; ++k) t += red[i * kWarpsW + k];
    v[i] = t;
  }
  __syncthreads();
}

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

// ------------------------------------------------------------------ Y build
// CTA = (key group g, 64-row block rb).  Warp w: rows 16 (w & 3) of the block,
// keys 4 (w >> 2) .. + 3 of the group, all z of each key (n_ao(Z) <= 32: four
// column tiles).  Per K step (one kept C pair t, 16 columns w of it):
//   As[NP][64][24]       C_XW rows (alpha, x), columns w
//   Bs[NP][8 * 32][24]   D_{W Z_i}[w][z] as rows (i, z), columns w
constexpr int kYRows = 64;
constexpr int kYS = 24;
size_t ybuild_w_smem(int np) { return (size_t)np * (kYRows + 256) * kYS * sizeof(uint16_t); }

template <int NP>
__global__ void __launch_bounds__(kWThreads) k_ybuild_w(DevPlan P, float* __restrict__ Yw, const int* ylist,
                                                        const int* gX, const int* gS, const int* gN, int RB) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* As = reinterpret_cast<uint16_t*>(smem);   // [NP][64][kYS]
  uint16_t* Bs = As + NP * kYRows * kYS;              // [NP][256][kYS]
  __shared__ int m_di[kMaxCPerAtom][8];
  __shared__ int m_step[2 * kMaxCPerAtom];
  __shared__ int s_key[8], s_zat[8], s_nz[8];
  __shared__ int s_nsteps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int g = blockIdx.x / RB, rb = blockIdx.x - g * RB;
  const int Xa = gX[g], kstart = gS[g], nk = gN[g];
  const int sX = P.species[Xa];
  const int mX = P.n_abf[sX], nX = P.n_ao[sX];
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
  // D block of every (kept C pair t, key i), or -1
  for (int e = threadIdx.x; e < nq * 8; e += blockDim.x) {
    const int t = e >> 3, i = e & 7;
    const int q = q0 + t;
    int di = -1;
    if (s_key[i] >= 0 && P.c_keep[q]) {
      const int* Rw = P.c_R + 3 * q;
      const int* Rz = P.y_R + 3 * s_key[i];
      di = dlut_get(P, P.c_j[q], s_zat[i], Rz[0] - Rw[0], Rz[1] - Rw[1], Rz[2] - Rw[2]);
      if (di >= 0 && P.Dkept[di] == 0.0) di = -1;
    }
    m_di[t][i] = di;
  }
  __syncthreads();
  if (threadIdx.x == 0) {   // K steps: (kept C pair with a D block among the keys, 16-column step)
    int n = 0;
    double fl = 0.0;
    for (int t = 0; t < nq; ++t) {
      bool any = false;
      const int nW = P.n_ao[P.species[P.c_j[q0 + t]]];
      for (int i = 0; i < 8; ++i)
        if (m_di[t][i] >= 0) {
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
  constexpr long long pA = kYRows * kYS, pB = 256 * kYS;
  for (int k = 0; k < nsteps; ++k) {
    const int t = m_step[k] >> 8, k0 = m_step[k] & 255;
    const int q = q0 + t;
    const int nW = P.n_ao[P.species[P.c_j[q]]];
    const double* C = P.Cst + P.c_off[q];
    __syncthreads();   // previous step's fragments read
    for (int e = threadIdx.x; e < kYRows * 16; e += blockDim.x) {
      const int r = e >> 4, c = e & 15;
      const int row = row0 + r, w = k0 + c;
      put_pieces<NP>(As, pA, r * kYS + c, (row < rows && w < nW) ? (float)C[(long long)row * nW + w] : 0.f);
    }
    for (int e = threadIdx.x; e < 256 * 16; e += blockDim.x) {
      const int rz = e >> 4, c = e & 15;
      const int i = rz >> 5, z = rz & 31, w = k0 + c;
      const int di = m_di[t][i];
      float v = 0.f;
      if (di >= 0 && w < nW && z < s_nz[i]) v = (float)P.Dval[P.Doff[di] + (long long)w * s_nz[i] + z];
      put_pieces<NP>(Bs, pB, rz * kYS + c, v);
    }
    __syncthreads();
    uint32_t af[NP][4];
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) ldm_x4(af[pp], As + pp * pA + (mt * 16 + (lane & 15)) * kYS + ((lane >> 4) << 3));
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      const int i = 4 * kh + ii;
      if (m_di[t][i] < 0) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        if (nt * 8 >= nz4[ii]) break;
        uint32_t bf[NP][2];
#pragma unroll
        for (int pp = 0; pp < NP; ++pp)
          ldm_x2(bf[pp], Bs + pp * pB + (i * 32 + nt * 8 + (lane & 7)) * kYS + (((lane >> 3) & 1) << 3));
        mma_split<NP>(acc[ii][nt], af, bf);
      }
    }
  }
  // Y (FP32) [alpha][x][z] = row (alpha, x), column z
#pragma unroll
  for (int ii = 0; ii < 4; ++ii) {
    const int key = s_key[4 * kh + ii];
    if (key < 0) continue;
    float* Y = Yw + P.y_off[key];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      if (nt * 8 >= nz4[ii]) break;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int row = row0 + mt * 16 + gid + ((c & 2) ? 8 : 0);
        const int z = nt * 8 + 2 * tig + (c & 1);
        if (row < rows && z < nz4[ii]) Y[(long long)row * nz4[ii] + z] = acc[ii][nt][c];
      }
    }
  }
}

// ------------------------------------------------------------------ term 1
// Shared memory (bf16 planes; strides are multiples of 8 elements with an
// odd count of 16-byte chunks, so that ldmatrix rows hit distinct banks):
//   Vs[NP][MA][MB + 8]   V_AB (rows alpha, columns beta; zero padded)
//   Ds[NP][40][40]       D_AB (rows a, columns b; zero padded)
//   Cs[NP][MA][KC + 8]   C_AF columns (a, f) of the current range of a
//   Us[NP][MB][KC + 8]   U of the same columns (rows beta)
struct T1W {
  int MA, MB, KC, da;
};

__host__ __device__ inline size_t term1w_smem(int np, int MA, int MB, int KC) {
  return (size_t)np * 2 * ((size_t)MA * (MB + 8) + 40 * 40 + (size_t)MA * (KC + 8) + (size_t)MB * (KC + 8));
}

template <int NP>
__global__ void __launch_bounds__(kWThreads) k_term1_w(DevPlan P, const float* __restrict__ Yw, const int* list,
                                                       int n_list, T1W S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[4 * kWarpsW];
  __shared__ double s_g[3];
  __shared__ int s_q;   // C pair whose grad C partials are in s_g
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int MA = S.MA, MB = S.MB;
  const int SV = MB + 8, SD = 40, SK = S.KC + 8;
  const long long pV = (long long)MA * SV, pD = 40 * SD, pC = (long long)MA * SK, pU = (long long)MB * SK;
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
    const double* Dg = P.Dval + P.Doff[P.v_didx[p]];
    __syncthreads();   // previous pair done with every buffer
    if (threadIdx.x == 0) {
      s_g[0] = s_g[1] = s_g[2] = 0.0;
      s_q = -1;
    }
    for (int e = threadIdx.x; e < MA * SV; e += blockDim.x) {
      const int al = e / SV, be = e - al * SV;
      put_pieces<NP>(Vs, pV, e, (al < mA && be < mB) ? (float)V[al * mB + be] : 0.f);
    }
    for (int e = threadIdx.x; e < 40 * SD; e += blockDim.x) {
      const int a = e / SD, bb = e - a * SD;
      put_pieces<NP>(Ds, pD, e, (a < nA && bb < nB) ? (float)Dg[a * nB + bb] : 0.f);
    }
    // U rows beyond n_abf(B) stay zero (they meet the zero V columns in Q)
    for (int e = threadIdx.x; e < (MB - mB) * SK; e += blockDim.x)
#pragma unroll
      for (int pp = 0; pp < NP; ++pp) Us[pp * pU + (long long)mB * SK + e] = 0;
    const RTiles rt(MAp, MBp);
    float racc[kRPairs][2][4];
#pragma unroll
    for (int i = 0; i < kRPairs; ++i)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int c = 0; c < 4; ++c) racc[i][h][c] = 0.f;
    double ev[4] = {0.0, 0.0, 0.0, 0.0};
    // E and g^V of the R run so far (FP32 dot, FP64 sum), then R restarts
    auto flush_r = [&]() {
      float evf[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < kRPairs; ++i) {
        const int pr = warp + kWarpsW * i;
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
        const float* Y = Yw + P.y_off[yc];             // [beta][b][f]
        const double* C = P.Cst + P.c_off[q];           // [alpha][a][f]
        const double* dC = P.dCst + 3 * P.c_off[q];
        const long long nc = (long long)mA * nA * nF;
        const int rowsU = mB * nF;
        float gq[3] = {0.f, 0.f, 0.f};
        for (int a0 = 0; a0 < nA; a0 += S.da) {
          const int dA = min(S.da, nA - a0);
          const int dcols = dA * nF, KCc = rup16(dcols);
          __syncthreads();   // the previous range's products are done with Cs and Us
          if (threadIdx.x == 0 && s_q >= 0 && s_q != q) {   // grad C partials of the previous F
            atomicAdd(&P.gC[3 * s_q + 0], -2.0 * s_g[0]);
            atomicAdd(&P.gC[3 * s_q + 1], -2.0 * s_g[1]);
            atomicAdd(&P.gC[3 * s_q + 2], -2.0 * s_g[2]);
            s_g[0] = s_g[1] = s_g[2] = 0.0;
          }
          if (threadIdx.x == 0) s_q = q;
          // C_AF columns (a, f), a in [a0, a0 + dA): contiguous in each row alpha
          for (int e = threadIdx.x; e < mA * KCc; e += blockDim.x) {
            const int al = e / KCc, c = e - al * KCc;
            put_pieces<NP>(Cs, pC, al * SK + c, c < dcols ? (float)C[(long long)al * nA * nF + a0 * nF + c] : 0.f);
          }
          // U columns past the range stay zero up to the 16-column step
          for (int e = threadIdx.x; e < mB * (KCc - dcols); e += blockDim.x) {
            const int be = e / (KCc - dcols), c = dcols + (e - be * (KCc - dcols));
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) Us[pp * pU + (long long)be * SK + c] = 0;
          }
          // U[(beta, f)][a] = sum_b Y[beta][b][f] D_AB[a][b]: rows (beta, f), one tile of 8 a
          for (int mt = warp; mt * 16 < rowsU; mt += kWarpsW) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            const int r0 = mt * 16 + gid, r1 = r0 + 8;
            const int be0 = r0 / nF, f0 = r0 - be0 * nF, be1 = r1 / nF, f1 = r1 - be1 * nF;
            for (int k0 = 0; k0 < KB; k0 += 16) {
              uint32_t af[NP][4], bf[NP][2];
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                const bool hi = h & 1;
                const int r = hi ? r1 : r0, be = hi ? be1 : be0, ff = hi ? f1 : f0;
                const int kc = k0 + 2 * tig + ((h & 2) ? 8 : 0);
                const bool in = r < rowsU;
                const float x0 = (in && kc < nB) ? Y[((long long)be * nB + kc) * nF + ff] : 0.f;
                const float x1 = (in && kc + 1 < nB) ? Y[((long long)be * nB + kc + 1) * nF + ff] : 0.f;
                uint32_t w[NP];
                split_pair<NP>(x0, x1, w);
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) af[pp][h] = w[pp];
              }
#pragma unroll
              for (int pp = 0; pp < NP; ++pp)
                ldm_x2(bf[pp], Ds + pp * pD + (a0 + (lane & 7)) * SD + k0 + (((lane >> 3) & 1) << 3));
              mma_split<NP>(acc, af, bf);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int r = (c & 2) ? r1 : r0;
              const int al = 2 * tig + (c & 1);
              if (r < rowsU && al < dA) {
                const int be = (c & 2) ? be1 : be0, ff = (c & 2) ? f1 : f0;
                put_pieces<NP>(Us, pU, be * SK + al * nF + ff, acc[c]);
              }
            }
          }
          __syncthreads();   // Cs and Us complete
          // R += C_AF . U^T (M = alpha, N = beta, K = this range's columns)
#pragma unroll
          for (int i = 0; i < kRPairs; ++i) {
            const int pr = warp + kWarpsW * i;
            if (pr >= rt.count()) break;
            const int mt = pr / rt.NTP, nt0 = 2 * (pr - mt * rt.NTP);
            gemm_pair_kk<NP>(racc[i], Cs, pC, SK, Us, pU, SK, mt, nt0, nt0 + 1 < rt.NT, KCc);
          }
          // Q = V_AB . U (M = alpha, N = columns, K = beta), dotted with grad C_AF
          {
            const int NTQ = rup8(dcols) >> 3, NPQ = (NTQ + 1) >> 1;
            const int npairs = (MAp >> 4) * NPQ;
            for (int pr = warp; pr < npairs; pr += kWarpsW) {
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
          if (lane == 0) atomicAdd(&s_g[c], (double)w);
        }
        fl += 2.0 * mB * nA * nB * nF + 4.0 * mA * mB * nA * nF;
        if (++nf % kFlushF == 0) flush_r();
      }
    }
    flush_r();
    block_sum_w<4>(ev, red);   // also orders the s_g additions before the flush below
    if (threadIdx.x == 0) {
      if (s_q >= 0) {
        atomicAdd(&P.gC[3 * s_q + 0], -2.0 * s_g[0]);
        atomicAdd(&P.gC[3 * s_q + 1], -2.0 * s_g[1]);
        atomicAdd(&P.gC[3 * s_q + 2], -2.0 * s_g[2]);
      }
      atomicAdd(&P.acc[ACC_E], -ev[0]);
      atomicAdd(&P.gV[3 * p + 0], -ev[1]);
      atomicAdd(&P.gV[3 * p + 1], -ev[2]);
      atomicAdd(&P.gV[3 * p + 2], -ev[3]);
      atomicAdd(&P.acc[ACC_F1], fl);
    }
  }
}

// ------------------------------------------------------------------ term 2
// Shared memory (bf16 planes):
//   Vs[NP][MA][MB + 8]          V_AB
//   Ya[NP][MA][KC + 8]          Y^{AB} columns (a, b), a in the current range
//   Yb[NP][MB][KC + 8]          Y^{BA} as [beta][(a, b)], same columns
//   Zs[NP][ZR][KZ + 8]          Z rows (alpha, a - a0), columns b (KZ = rup16 max n_ao)
//   gF[3 * kMaxCPerAtom]        FP64 grad C partials per C slot of A
//   fdi[kMaxCPerAtom]           D_FB block per C slot of A (or -1)
struct T2W {
  int MA, MB, KC, da, ZR, KZ;
};

__host__ __device__ inline size_t term2w_smem(int np, int MA, int MB, int KC, int ZR, int KZ) {
  return (size_t)np * 2 *
             ((size_t)MA * (MB + 8) + (size_t)MA * (KC + 8) + (size_t)MB * (KC + 8) + (size_t)ZR * (KZ + 8)) +
         (size_t)3 * kMaxCPerAtom * sizeof(double) + (size_t)kMaxCPerAtom * sizeof(int);
}

template <int NP>
__global__ void __launch_bounds__(kWThreads) k_term2_w(DevPlan P, const float* __restrict__ Yw, const int* list,
                                                       int n_list, T2W S) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[4 * kWarpsW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
  const int MA = S.MA, MB = S.MB;
  const int SV = MB + 8, SK = S.KC + 8, SZ = S.KZ + 8;
  const long long pV = (long long)MA * SV, pA = (long long)MA * SK, pB = (long long)MB * SK, pZ = (long long)S.ZR * SZ;
  double* gF = reinterpret_cast<double*>(smem);
  int* fdi = reinterpret_cast<int*>(gF + 3 * kMaxCPerAtom);
  uint16_t* Vs = reinterpret_cast<uint16_t*>(fdi + kMaxCPerAtom);
  uint16_t* Ya = Vs + NP * pV;
  uint16_t* Yb = Ya + NP * pA;
  uint16_t* Zs = Yb + NP * pB;
  for (int kk = blockIdx.x; kk < n_list; kk += gridDim.x) {
    const int p = list[kk];
    const int A = P.v_home[p], b = P.v_j[p];
    const int* Rb = P.v_R + 3 * p;
    const int sA = P.species[A], sB = P.species[b];
    const int nA = P.n_ao[sA], nB = P.n_ao[sB], mA = P.n_abf[sA], mB = P.n_abf[sB];
    const int MAp = rup16(mA), MBp = rup16(mB), KB = rup16(nB);
    const int y1 = ylut_get(P, A, b, Rb[0], Rb[1], Rb[2]);
    const int y2 = ylut_get(P, b, A, -Rb[0], -Rb[1], -Rb[2]);
    const float* Yab = Yw + P.y_off[y1];   // [alpha][a][b]
    const float* Yba = Yw + P.y_off[y2];   // [beta][b][a]
    const double* V = P.Vst + P.v_off[p];
    const int nvb = mA * mB, nab = nA * nB;
    const int q0 = P.c_ptr[A], nq = P.c_ptr[A + 1] - q0;
    __syncthreads();   // previous pair done with every buffer
    for (int t = threadIdx.x; t < nq; t += blockDim.x) {
      const int q = q0 + t;
      int di = -1;
      if (P.c_keep[q]) {
        const int* Rf = P.c_R + 3 * q;
        di = dlut_get(P, P.c_j[q], b, Rb[0] - Rf[0], Rb[1] - Rf[1], Rb[2] - Rf[2]);
        if (di >= 0 && P.Dkept[di] == 0.0) di = -1;
      }
      fdi[t] = di;
      gF[3 * t] = gF[3 * t + 1] = gF[3 * t + 2] = 0.0;
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
    float racc[kRPairs][2][4];
#pragma unroll
    for (int i = 0; i < kRPairs; ++i)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int c = 0; c < 4; ++c) racc[i][h][c] = 0.f;
    double fl = 4.0 * mA * mB * nA * nB;
    for (int a0 = 0; a0 < nA; a0 += S.da) {
      const int dA = min(S.da, nA - a0);
      const int dcols = dA * nB, KCc = rup16(dcols);
      const int zrows = mA * S.da;
      __syncthreads();   // the previous range is done with Ya, Yb and Zs
      for (int e = threadIdx.x; e < mA * KCc; e += blockDim.x) {
        const int al = e / KCc, c = e - al * KCc;
        put_pieces<NP>(Ya, pA, al * SK + c, c < dcols ? Yab[(long long)al * nab + a0 * nB + c] : 0.f);
      }
      for (int e = threadIdx.x; e < mB * KCc; e += blockDim.x) {
        const int be = e / KCc, c = e - be * KCc;
        float v = 0.f;
        if (c < dcols) {
          const int al = c / nB, bb = c - al * nB;
          v = Yba[(long long)be * nab + bb * nA + a0 + al];
        }
        put_pieces<NP>(Yb, pB, be * SK + c, v);
      }
      // Z columns b past n_ao(B) stay zero up to the 16-column step (K of Q2)
      for (int e = threadIdx.x; e < zrows * (KB - nB); e += blockDim.x) {
        const int r = e / (KB - nB), c = nB + (e - r * (KB - nB));
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) Zs[pp * pZ + (long long)r * SZ + c] = 0;
      }
      __syncthreads();
      // R2 += Y^{AB} . Y^{BA} (M = alpha, N = beta, K = (a, b) of the range)
#pragma unroll
      for (int i = 0; i < kRPairs; ++i) {
        const int pr = warp + kWarpsW * i;
        if (pr >= rt.count()) break;
        const int mt = pr / rt.NTP, nt0 = 2 * (pr - mt * rt.NTP);
        gemm_pair_kk<NP>(racc[i], Ya, pA, SK, Yb, pB, SK, mt, nt0, nt0 + 1 < rt.NT, KCc);
      }
      // Z = V_AB . Y^{BA} (M = alpha, N = (a, b), K = beta) -> Zs rows (alpha, a - a0)
      {
        const int NTZ = rup8(dcols) >> 3, NPZ = (NTZ + 1) >> 1;
        const int npairs = (MAp >> 4) * NPZ;
        for (int pr = warp; pr < npairs; pr += kWarpsW) {
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
                const int a = n / nB, bb = n - a * nB;
                put_pieces<NP>(Zs, pZ, (al * S.da + a) * SZ + bb, acc[h][c]);
              }
            }
        }
      }
      __syncthreads();   // Zs complete
      // per C pair (A,F) with D_FB kept: Q2[(alpha, a)][f] = sum_b Z[(alpha, a)][b] D_FB[f][b]
      const int MTZ = (zrows + 15) >> 4;
      for (int t = 0; t < nq; ++t) {
        const int di = fdi[t];
        if (di < 0) continue;
        const int q = q0 + t;
        const int nF = P.n_ao[P.species[P.c_j[q]]];
        const double* Dfb = P.Dval + P.Doff[di];   // [f][b]
        const double* dC = P.dCst + 3 * P.c_off[q];
        const long long nc = (long long)mA * nA * nF;
        const int NTF = rup8(nF) >> 3;
        float gq[3] = {0.f, 0.f, 0.f};
        if (warp < MTZ) {
          // B fragments of D_FB (K = b, N = f), this warp's for every m tile
          uint32_t bfr[4][2][NP][2];
#pragma unroll
          for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int ff = nt * 8 + gid, kc = ks * 16 + 2 * tig + (h ? 8 : 0);
                const bool in = nt < NTF && ff < nF;
                const float x0 = (in && kc < nB) ? (float)Dfb[ff * nB + kc] : 0.f;
                const float x1 = (in && kc + 1 < nB) ? (float)Dfb[ff * nB + kc + 1] : 0.f;
                uint32_t w[NP];
                split_pair<NP>(x0, x1, w);
#pragma unroll
                for (int pp = 0; pp < NP; ++pp) bfr[nt][ks][pp][h] = w[pp];
              }
          for (int mt = warp; mt < MTZ; mt += kWarpsW) {
            float acc[4][4];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[nt][c] = 0.f;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              if (ks * 16 >= KB) break;
              uint32_t af[NP][4];
#pragma unroll
              for (int pp = 0; pp < NP; ++pp)
                ldm_x4(af[pp], Zs + pp * pZ + (long long)(mt * 16 + (lane & 15)) * SZ + ks * 16 + ((lane >> 4) << 3));
#pragma unroll
              for (int nt = 0; nt < 4; ++nt) {
                if (nt >= NTF) break;
                mma_split<NP>(acc[nt], af, bfr[nt][ks]);
              }
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
              if (nt >= NTF) break;
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const int r = mt * 16 + gid + ((c & 2) ? 8 : 0);
                const int ff = nt * 8 + 2 * tig + (c & 1);
                const int al = r / S.da, a = a0 + (r - al * S.da);
                if (r < zrows && a < a0 + dA && ff < nF) {
                  const long long ci = ((long long)al * nA + a) * nF + ff;
                  const float v = acc[nt][c];
                  gq[0] = fmaf((float)dC[ci], v, gq[0]);
                  gq[1] = fmaf((float)dC[nc + ci], v, gq[1]);
                  gq[2] = fmaf((float)dC[2 * nc + ci], v, gq[2]);
                }
              }
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float w = warp_sum_f(gq[c]);
          if (lane == 0 && w != 0.f) atomicAdd(&gF[3 * t + c], (double)w);
        }
        if (a0 == 0 && threadIdx.x == 0) fl += 2.0 * mA * nA * nB * nF;
      }
    }
    // E and g^V from R2
    double ev[4] = {0.0, 0.0, 0.0, 0.0};
    {
      float evf[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < kRPairs; ++i) {
        const int pr = warp + kWarpsW * i;
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
    block_sum_w<4>(ev, red);   // also orders the gF additions before the flush below
    for (int t = threadIdx.x; t < nq; t += blockDim.x) {
      if (gF[3 * t] != 0.0 || gF[3 * t + 1] != 0.0 || gF[3 * t + 2] != 0.0) {
        const int q = q0 + t;
        atomicAdd(&P.gC[3 * q + 0], -2.0 * gF[3 * t + 0]);
        atomicAdd(&P.gC[3 * q + 1], -2.0 * gF[3 * t + 1]);
        atomicAdd(&P.gC[3 * q + 2], -2.0 * gF[3 * t + 2]);
      }
    }
    if (threadIdx.x == 0) {
      atomicAdd(&P.acc[ACC_E], -ev[0]);
      atomicAdd(&P.gV[3 * p + 0], -ev[1]);
      atomicAdd(&P.gV[3 * p + 1], -ev[2]);
      atomicAdd(&P.gV[3 * p + 2], -ev[3]);
      atomicAdd(&P.acc[ACC_F2], fl);
    }
  }
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
    const int ZR = (maxABF * da + 15) / 16 * 16;
    if (term2w_smem(np, w.MA, w.MB, KC, ZR, w.KZ) <= limit) {
      w.t2_da = da;
      w.t2_KC = KC;
      w.t2_ZR = ZR;
      w.smem_t2 = term2w_smem(np, w.MA, w.MB, KC, ZR, w.KZ);
      break;
    }
  }
  // R tiles: (MA / 16) x (MB / 16) pairs over the 8 warps, kRPairs each
  w.ok = w.t1_da > 0 && w.t2_da > 0 && (w.MA / 16) * (w.MB / 16) <= kWarpsW * kRPairs && maxAO <= 32;
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
  } else {
    one((const void*)k_ybuild_w<3>);
    one((const void*)k_term1_w<3>);
    one((const void*)k_term2_w<3>);
  }
  return e;
}

cudaError_t launch_ybuild_w(const DevPlan& P, int np, float* Yw, const int* ylist, const int* gX, const int* gS,
                            const int* gN, int ngroups, int RB, cudaStream_t s) {
  if (ngroups <= 0) return cudaSuccess;
  const long long grid = (long long)ngroups * RB;
  const size_t smem = ybuild_w_smem(np);
  if (np == 2) k_ybuild_w<2><<<(unsigned)grid, kWThreads, smem, s>>>(P, Yw, ylist, gX, gS, gN, RB);
  else k_ybuild_w<3><<<(unsigned)grid, kWThreads, smem, s>>>(P, Yw, ylist, gX, gS, gN, RB);
  ++g_wide_launches;
  return cudaGetLastError();
}

cudaError_t launch_term1_w(const DevPlan& P, int np, const float* Yw, const int* list, int n, const WideShapes& w,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const T1W S{w.MA, w.MB, w.t1_KC, w.t1_da};
  const int grid = grid_cap(n, 1 << 20);
  if (np == 2) k_term1_w<2><<<grid, kWThreads, w.smem_t1, s>>>(P, Yw, list, n, S);
  else k_term1_w<3><<<grid, kWThreads, w.smem_t1, s>>>(P, Yw, list, n, S);
  ++g_wide_launches;
  return cudaGetLastError();
}

cudaError_t launch_term2_w(const DevPlan& P, int np, const float* Yw, const int* list, int n, const WideShapes& w,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const T2W S{w.MA, w.MB, w.t2_KC, w.t2_da, w.t2_ZR, w.KZ};
  const int grid = grid_cap(n, 1 << 20);
  if (np == 2) k_term2_w<2><<<grid, kWThreads, w.smem_t2, s>>>(P, Yw, list, n, S);
  else k_term2_w<3><<<grid, kWThreads, w.smem_t2, s>>>(P, Yw, list, n, S);
  ++g_wide_launches;
  return cudaGetLastError();
}

}  // namespace hfx
