// First exchange product of the HFX force/stress on the 5th-generation tensor
// cores (tcgen05 MMAs with accumulators in tensor memory), split-bf16 operands.
//
// For a kept C pair (A,F) (an "item") and its kept V pairs (A,B), the first
// product of Eq. exx_expand, factorised through Y^{BF} = sum_W C_BW D_WF:
//   U_B[beta][(f,a)] = sum_b Y^{BF}[f][beta][b] D_AB[a][b]   (CUDA cores, FP32)
//   R_B = C_AF . U_B^T        (M = alpha, N = beta, K = (f,a))  -> g^V_AB = -<grad V_AB, R_B>
//                             (two U pieces per instruction, N = 128: R is the sum of two 64-column blocks)
//   Q  += V_AB . U_B          (M = alpha, N = (f,a), K = beta)  -> E = -<C_AF, Q>, g^C_AF = -2 <grad C_AF, Q>
// (E through Q: <V_AB, C U^T> = <C, V_AB U>, so the per-B epilogue carries
// only the three gradient planes of V.)
//
// Column order (f,a) = 16 f + a with a padded to 16: a U row of one f is two
// whole core matrices, so the CUDA cores write U with 8-byte stores and no
// bank conflicts.  All matrices sit in shared memory in the no-swizzle
// core-matrix order (8 rows x 16 bytes); U serves R as a K-major B operand
// and Q as an MN-major B operand without a second copy.
//
// Warp roles (16 warps, one CTA per SM, persistent over items):
//   warp 0      Y producer: bulk copies of runs of up to FS rows Y^{BF}[f]
//               (FP32, never crossing a U chunk) into a ring of NS slots
//   warp 1      scheduler and producer: takes items from a global counter
//               (dynamic load balance), hands them to the other roles through
//               a ring two items ahead, and copies C (per item), D_AB (FP32)
//               and V_AB pieces (per B)
//   warp 2      tensor-memory owner; lane 0 issues the R products
//   warp 3      lane 0 issues the Q products (a second issuing thread on
//               another SMSP: one thread issues an MMA only every ~50 cycles)
//   warps 4-7   epilogue: R -> g^V per B; Q -> E, g^C per run of B
//   warps 8-15  U: one thread per (beta, 4 columns a) of each f
// All hand-offs are mbarriers (bounded waits; a timeout sets the error flag
// and every role stops), no block barrier inside the pipeline.
#include <algorithm>
#include <atomic>
#include <mutex>

#include "hfx_accum.cuh"
#include "hfx_device.cuh"
#include "hfx_model.cuh"

namespace hfx {
namespace {

using namespace dev;

std::atomic<long long> g_t1u_launches{0};

constexpr int kThreads = 512;
constexpr int kWarpY = 0, kWarpV = 1, kWarpM = 2, kWarpQ = 3, kWarpE = 4, kWarpU = 8;
constexpr int kNE = 4, kNU = 8;
constexpr int kItemRing = 4;
constexpr int kItemReaders = 3 + kNE + kNU;   // Y, R issuer, Q issuer, epilogue warps, U warps
constexpr int kMaxNS = 16;
constexpr int kRCol = 256;   // tensor-memory column of the first R accumulator (Q sits at column 0)
constexpr int kRCols = 128;  // columns of one R accumulator: two 64-column blocks, R = block 0 + block 1

__device__ __forceinline__ bool aborted(const volatile int* f) { return *f != 0; }

// Every lane waits (bounded); the result is the same on all lanes.
__device__ __forceinline__ bool wait_all(uint32_t mbar, uint32_t parity) {
  return __all_sync(0xffffffffu, mbar_wait(mbar, parity)) != 0;
}

// ------------------------------------------------------------ operand stores
// Order in which the epilogue warps load a 64-row FP32 plane (C, grad C,
// grad V): epilogue warp qd = alpha >> 4 holds row alpha in lane
// (alpha & 15) + 16 h and reads columns 32 j + 16 h + 4 t .. + 3 as one
// float4, so that for each (j, t) a warp's 32 loads are 512 consecutive
// bytes; element (alpha, col) sits at float
// ((((j * 4 + t) * 4 + qd) * 32 + lane) << 2) + (col & 3).  ep_at gives the
// (alpha, col) stored at float w (the stores are written in storage order).
__device__ __forceinline__ void ep_at(int w, int& alpha, int& col) {
  const int k = w & 3, l = (w >> 2) & 31, qd = (w >> 7) & 3, t = (w >> 9) & 3, j = w >> 11;
  alpha = qd * 16 + (l & 15);
  col = 32 * j + 16 * (l >> 4) + 4 * t + k;
}

// Item kk (C pair q = list[kk]): NP bf16 pieces of C_AF as [alpha (64)][(f,a) (KP)]
// in core-matrix order (8-row groups of KP/8 core matrices), then C and
// grad C in FP32 as four planes of 64 x KP32 (KP rounded up to 32) in
// epilogue load order (ep_at).  Zero padded.  Each plane of the C pair
// ([(alpha,a)][f]) is evaluated from the block model into shared memory as
// FP32; the outputs are written in storage order, four elements per thread.
constexpr int kCStoreSmem = 64 * 16 * 16 * 4;   // one plane of n_abf <= 64, n_ao <= 16

template <int NP>
__global__ void k_t1u_cstore(DevPlan P, T1UPlan U, const int* list, int n) {
  extern __shared__ float cs[];
  const int KP = U.KP, KP32 = t1u_kp32(KP), PL = 64 * KP32;
  for (int kk = blockIdx.x; kk < n; kk += gridDim.x) {
    const int q = list[kk];
    const int A = P.c_home[q], F = P.c_j[q];
    const int sA = P.species[A];
    const int nA = P.n_ao[sA], mA = P.n_abf[sA], nF = P.n_ao[P.species[F]];
    const int ncq = mA * nA * nF;
    uint16_t* out = U.Cu + (long long)kk * U.cu_blk;
    float* pl = reinterpret_cast<float*>(out + (long long)NP * 64 * KP);
    float scf[8];   // C = G f + G' fa, grad C = G g + G' ga (block model, FP32 as k_cpieces)
#pragma unroll
    for (int k = 0; k < 8; ++k) scf[k] = (float)P.c_sc[8 * (long long)q + k];
    const long long go = P.G_off[sA * P.S + P.species[F]];
    for (int c = 0; c < 4; ++c) {
      __syncthreads();
      for (int e = threadIdx.x; e < ncq; e += blockDim.x) cs[e] = model::c_value_f(P, scf, go, e, c);
      __syncthreads();
      auto val = [&](int al, int col) -> float {
        const int f = col >> 4, a = col & 15;
        return (al < mA && col < KP && f < nF && a < nA) ? cs[(al * nA + a) * nF + f] : 0.f;
      };
      if (c == 0) {
        // pieces: core-matrix element t -> (alpha, col), four consecutive columns per thread
        for (int t4 = threadIdx.x; t4 < 16 * KP; t4 += blockDim.x) {
          const int t = 4 * t4;
          const int g8 = t / (KP * 8), rem = t - g8 * KP * 8;
          const int al = g8 * 8 + ((rem >> 3) & 7), col = (rem >> 6) * 8 + (rem & 7);
          const float x[4] = {val(al, col), val(al, col + 1), val(al, col + 2), val(al, col + 3)};
          uint2 pc[NP];
          split4<NP>(x, pc);
#pragma unroll
          for (int pp = 0; pp < NP; ++pp) *reinterpret_cast<uint2*>(out + (long long)pp * 64 * KP + t) = pc[pp];
        }
      }
      for (int w4 = threadIdx.x; w4 < PL / 4; w4 += blockDim.x) {   // FP32 plane c, storage order
        int al, col;
        ep_at(4 * w4, al, col);
        *reinterpret_cast<float4*>(pl + (long long)c * PL + 4 * w4) =
            make_float4(val(al, col), val(al, col + 1), val(al, col + 2), val(al, col + 3));
      }
    }
  }
}

// Every needed V pair p = list[k], in one pass: V and grad V evaluated once
// from the block model into shared memory (FP32), then
//   the warp-level second product's store X.Vm at vm_off[p] (unless X.Vz is
//   set): NP bf16 planes [alpha][rup16(n_abf(B))] and V, grad V in FP32
//   [4][n_abf(A) n_abf(B)];
//   for the pairs of the first product (any bit of v_mask), the tcgen05
//   store U.Vu at t1_idx[p]: NP pieces [alpha 64][beta 64] in core-matrix
//   order and grad V in three planes in epilogue load order (ep_at);
//   for the pairs of the second product (v_t2), with X.Vz set, the store of
//   k_t2_umma at t2_slot[p]: the same pieces and V, grad V in four planes.
// Outputs are written in storage order, four elements per thread.
constexpr int kVStoreSmem = 4 * 64 * 64 * 4;

template <int NP>
__global__ void k_vstores(DevPlan P, MixPlan X, T1UPlan U, const int* list, int n) {
  extern __shared__ float vsm[];   // [4][mA * mB]: V, grad V
  for (int k = blockIdx.x; k < n; k += gridDim.x) {
    const int p = list[k];
    const int sA = P.species[P.v_home[p]], sB = P.species[P.v_j[p]];
    const int mA = P.n_abf[sA], mB = P.n_abf[sB], MB = rup16(mB), nv = mA * mB;
    double h, g[3];
    model::v_pair(P, p, h, g);   // V = M h, grad V = M g (block model), in FP32
    const float hf = (float)h, g0 = (float)g[0], g1 = (float)g[1], g2 = (float)g[2];
    const float* M = P.Mf + P.M_off[sA * P.S + sB];
    __syncthreads();
    for (int e = threadIdx.x; e < nv; e += blockDim.x) {
      const float m = M[e];
      vsm[e] = m * hf;
      vsm[nv + e] = m * g0;
      vsm[2 * nv + e] = m * g1;
      vsm[3 * nv + e] = m * g2;
    }
    __syncthreads();
    // second-product store of the warp-level R2 / Z kernel (none with the
    // tcgen05 one, X.Vz: nothing reads it then)
    if (!X.Vz) {
      uint16_t* out = X.Vm + X.vm_off[p];
      for (int e4 = threadIdx.x; e4 < mA * MB / 4; e4 += blockDim.x) {
        const int e = 4 * e4, al = e / MB, be = e - al * MB;
        float x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = be + j < mB ? vsm[al * mB + be + j] : 0.f;
        uint2 pc[NP];
        split4<NP>(x, pc);
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) *reinterpret_cast<uint2*>(out + (long long)pp * mA * MB + e) = pc[pp];
      }
      float* v32 = reinterpret_cast<float*>(out + (long long)NP * mA * MB);
      for (int e = threadIdx.x; e < 4 * nv; e += blockDim.x) v32[e] = vsm[e];
    }
    // first-product store
    bool t1 = false;
#pragma unroll
    for (int w = 0; w < kMaskWords; ++w) t1 = t1 || P.v_mask[(long long)p * kMaskWords + w] != 0u;
    // the tcgen05 stores: the first product's (U.Vu, per first-product pair:
    // pieces and the three grad V planes) and the second product's (X.Vz, per
    // second-product pair: pieces and the four planes V, grad V)
    for (int st = 0; st < 2; ++st) {
      uint16_t* vu = nullptr;
      if (st == 0 && U.Vu && t1) vu = U.Vu + U.t1_idx[p] * U.vu_blk;
      if (st == 1 && X.Vz && P.v_t2[p]) vu = X.Vz + X.t2_slot[p] * X.vz_blk;
      if (!vu) continue;
      for (int t4 = threadIdx.x; t4 < 1024; t4 += blockDim.x) {   // core-matrix order, 4 columns per thread
        const int t = 4 * t4;
        const int al = ((t >> 9) << 3) + ((t >> 3) & 7), be = (((t >> 6) & 7) << 3) + (t & 7);
        float x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = (al < mA && be + j < mB) ? vsm[al * mB + be + j] : 0.f;
        uint2 pc[NP];
        split4<NP>(x, pc);
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) *reinterpret_cast<uint2*>(vu + pp * 4096 + t) = pc[pp];
      }
      float* pl = reinterpret_cast<float*>(vu + NP * 4096);
      const int c0 = st == 0 ? 1 : 0;   // first plane: grad V (first product) or V (second)
      for (int w4 = threadIdx.x; w4 < (4 - c0) * 1024; w4 += blockDim.x) {   // epilogue load order
        const int c = c0 + (w4 >> 10);
        int al, be;
        ep_at(4 * (w4 & 1023), al, be);
        float4 o;
        o.x = (al < mA && be < mB) ? vsm[c * nv + al * mB + be] : 0.f;
        o.y = (al < mA && be + 1 < mB) ? vsm[c * nv + al * mB + be + 1] : 0.f;
        o.z = (al < mA && be + 2 < mB) ? vsm[c * nv + al * mB + be + 2] : 0.f;
        o.w = (al < mA && be + 3 < mB) ? vsm[c * nv + al * mB + be + 3] : 0.f;
        *reinterpret_cast<float4*>(pl + 4 * w4) = o;
      }
    }
  }
}

// D block k as FP32 [16][16], zero padded; the four 16-byte chunks of row a
// are permuted by (a >> 2) & 3, so that rows 4 apart read the same chunk from
// different banks.
__global__ void k_t1u_dstore(DevPlan P, float* Df) {
  for (long long k = blockIdx.x; k < P.n_d; k += gridDim.x) {
    const int na = P.n_ao[P.species[P.Didx[5 * k]]], nb = P.n_ao[P.species[P.Didx[5 * k + 1]]];
    const double* src = P.Dval + P.Doff[k];
    for (int e = threadIdx.x; e < 256; e += blockDim.x) {
      const int a = e >> 4, b = e & 15;
      Df[k * 256 + a * 16 + (((b >> 2) ^ ((a >> 2) & 3)) << 2) + (b & 3)] =
          (a < na && b < nb) ? (float)src[a * nb + b] : 0.f;
    }
  }
}

// ------------------------------------------------- longest-first item order
// Items run on a dynamic queue; handing out the ones with the most kept B
// first keeps the last items short, so the SMs finish together.  Counting
// sort on the bucket (kLptBuckets - 1 - min(qcnt, kLptBuckets - 1)); the
// order of equal keys is not fixed (it does not change any item's result).
// With asc = 1 the same sort orders the items by key[q] ascending (the
// order by F: items of one F, which share many Y^{BF} blocks, run together).
__device__ __forceinline__ int lpt_bucket(const int* key, int q, int asc) {
  const int k = min(key[q], kLptBuckets - 1);
  return asc ? k : kLptBuckets - 1 - k;
}

__global__ void k_lpt_hist(const int* key, int asc, const int* list, const long long* n_dev, int* hist) {
  const int n = (int)*n_dev;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicAdd(&hist[lpt_bucket(key, list[i], asc)], 1);
}

// Exclusive scan of the histogram, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_lpt_scan(int* hist) {
  constexpr int kPer = kLptBuckets / 1024;
  __shared__ int part[1024];
  int v[kPer], t = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    v[j] = hist[threadIdx.x * kPer + j];
    t += v[j];
  }
  part[threadIdx.x] = t;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int add = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  int run = part[threadIdx.x] - t;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    hist[threadIdx.x * kPer + j] = run;
    run += v[j];
  }
}

__global__ void k_lpt_scatter(const int* key, int asc, const int* list, const long long* n_dev, int* hist, int* out) {
  const int n = (int)*n_dev;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int q = list[i];
    out[atomicAdd(&hist[lpt_bucket(key, q, asc)], 1)] = q;
  }
}

// ------------------------------------------------------------------- kernel
template <int NP>
__global__ void __launch_bounds__(kThreads, 1)
    k_t1_umma(DevPlan P, MixPlan X, T1UPlan U, const int* qlist, int n_list, int* work, int* err) {
  const int KP = U.KP, KP32 = t1u_kp32(KP), NF = KP >> 4, FH = (NF + 1) >> 1, NS = U.NS, SEG = U.seg, FS = U.FS;
  const int SLOT = FS * 64 * 16;                 // floats of one Y slot (FS rows f of up to 64 beta)
  constexpr int NPROD = NP * (NP + 1) / 2;       // piece products (i, j) with i + j < NP
  const uint32_t CPB = 64u * KP * 2u;            // bytes of one piece of C or U
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint16_t* Cs = reinterpret_cast<uint16_t*>(smem_raw);
  uint16_t* Us = Cs + (size_t)NP * 64 * KP;
  uint16_t* Vs = Us + (size_t)NP * 64 * KP;
  float* Ds = reinterpret_cast<float*>(Vs + NP * 4096);
  float* Ys = Ds + 2 * 256;
  __shared__ __align__(8) uint64_t b_yf[kMaxNS], b_ye[kMaxNS], b_cf, b_ce, b_vf, b_ve, b_df[2], b_de[2], b_uf[2],
      b_ue[2], b_rf[2], b_re[2], b_qf, b_qe, b_if[kItemRing], b_ie[kItemRing];
  __shared__ int s_item[kItemRing];
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  volatile int* abort_flag = &s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto sa = [](const void* p) { return (uint32_t)__cvta_generic_to_shared(p); };
  const uint32_t yf = sa(b_yf), ye = sa(b_ye), cf = sa(&b_cf), ce = sa(&b_ce), vf = sa(&b_vf), ve = sa(&b_ve),
                 df = sa(b_df), de = sa(b_de), uf = sa(b_uf), ue = sa(b_ue), rf = sa(b_rf), re = sa(b_re),
                 qf = sa(&b_qf), qe = sa(&b_qe), itf = sa(b_if), ite = sa(b_ie);
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < NS; ++s) {
      mbar_init(yf + 8 * s, 1);
      mbar_init(ye + 8 * s, kNU);
    }
    mbar_init(cf, 1);
    mbar_init(ce, 1);
    mbar_init(vf, 1);
    mbar_init(ve, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(df + 8 * s, 1);
      mbar_init(de + 8 * s, kNU);
      mbar_init(uf + 8 * s, kNU);
      mbar_init(ue + 8 * s, 2);   // released by both issuers
      mbar_init(rf + 8 * s, 1);
      mbar_init(re + 8 * s, kNE);
    }
    mbar_init(qf, 1);
    mbar_init(qe, kNE);
    for (int s = 0; s < kItemRing; ++s) {
      mbar_init(itf + 8 * s, 1);
      mbar_init(ite + 8 * s, kItemReaders);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == kWarpM) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sa(&tmem_base)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t T = tmem_base;
  // Next item of the ring for a role (one reader per warp; lane 0 releases
  // the slot).  n_list marks the end.  Every lane of the warp calls it.
  auto next_item = [&](uint32_t& k) -> int {
    const int s = k & (kItemRing - 1);
    int kk = n_list;
    if (wait_all(itf + 8 * s, (k / kItemRing) & 1)) kk = *reinterpret_cast<volatile int*>(&s_item[s]);
    else *abort_flag = 1;
    __syncwarp();
    if (lane == 0) mbar_arrive(ite + 8 * s);
    ++k;
    return kk;
  };

  if (warp == kWarpY) {
    // ---------------------------------------------------------- Y producer
    uint32_t ys = 0, ik = 0;
    for (int kk = next_item(ik); kk < n_list && !aborted(abort_flag); kk = next_item(ik)) {
      const int q = qlist[kk];
      const int F = P.c_j[q];
      const int nF = P.n_ao[P.species[F]];
      const int* Rf = P.c_R + 3 * q;
      const long long b0 = X.qoff[q];
      const int nbt = X.qcnt[q];
      for (int i0 = 0; i0 < nbt && !aborted(abort_flag); i0 += 32) {
        long long yo = 0;
        int mB = 0;
        if (i0 + lane < nbt) {
          const int p = X.blist[b0 + i0 + lane];
          const int b = P.v_j[p];
          const int* Rb = P.v_R + 3 * p;
          const int yc = ylut_get(P, b, F, Rf[0] - Rb[0], Rf[1] - Rb[1], Rf[2] - Rb[2]);
          yo = yc >= 0 ? P.y_off[yc] / NP : -1;
          mB = P.n_abf[P.species[b]];
        }
        const int nb = min(32, nbt - i0);
        for (int j = 0; j < nb; ++j) {
          const long long yoj = __shfl_sync(0xffffffffu, yo, j);
          const int mBj = __shfl_sync(0xffffffffu, mB, j);
          if (lane == 0 && !aborted(abort_flag)) {
            if (yoj < 0) *abort_flag = 1;   // a kept triplet always has its Y block
            // runs [fa, fb) of at most FS rows, within each U chunk, rows f < nF only
            for (int c = 0; c < 2 && !aborted(abort_flag); ++c) {
              const int e = min(c ? NF : FH, nF);
              for (int fa = c ? FH : 0; fa < e && !aborted(abort_flag); fa += FS) {
                const int fb = min(fa + FS, e);
                const int s = (int)(ys % NS);
                if (ys >= (uint32_t)NS && !mbar_wait(ye + 8 * s, ((ys / NS) - 1) & 1)) {
                  *abort_flag = 1;
                  break;
                }
                const uint32_t bytes = (uint32_t)((fb - fa) * mBj) * 64u;
                mbar_expect_tx(yf + 8 * s, bytes);
                bulk_g2s(sa(Ys + s * SLOT), U.Yf + yoj + (long long)fa * mBj * 16, bytes, yf + 8 * s);
                ++ys;
              }
            }
          }
          __syncwarp();
        }
      }
    }
    if (lane == 0)   // copies in flight land before the CTA leaves
      for (int s = 0; s < NS; ++s) {
        const uint32_t n = ys / NS + ((uint32_t)s < ys % NS ? 1u : 0u);
        if (n) mbar_wait(yf + 8 * s, (n - 1) & 1);
      }
  } else if (warp == kWarpV) {
    // -------------------------------------- scheduler, C, D and V producer
    // Lane 0 publishes item indices two items ahead of this warp's own
    // position (a slot is reused once every reader has taken its item).
    uint32_t pub = 0;
    bool pub_done = false;
    auto publish = [&]() {
      const int s = pub & (kItemRing - 1);
      if (pub >= kItemRing && !mbar_wait(ite + 8 * s, ((pub / kItemRing) - 1) & 1)) {
        *abort_flag = 1;
        s_item[s] = n_list;   // best effort: readers also stop on the flag
        pub_done = true;
        return;
      }
      int kk = aborted(abort_flag) ? n_list : atomicAdd(work, 1);
      if (kk > n_list) kk = n_list;
      s_item[s] = kk;
      mbar_arrive(itf + 8 * s);
      ++pub;
      if (kk >= n_list) pub_done = true;
    };
    if (lane == 0) {
      publish();
      if (!pub_done) publish();
    }
    __syncwarp();
    uint32_t vb = 0, db = 0, it = 0, ca = 0, own = 0;
    auto own_item = [&]() -> int {
      int kk = n_list;
      if (lane == 0 && own < pub) kk = *reinterpret_cast<volatile int*>(&s_item[own & (kItemRing - 1)]);
      ++own;
      return __shfl_sync(0xffffffffu, kk, 0);
    };
    for (int kk = own_item(); kk < n_list && !aborted(abort_flag); kk = own_item(), ++it) {
      const int q = qlist[kk];
      const long long b0 = X.qoff[q];
      const int nbt = X.qcnt[q];
      if (lane == 0) {
        if (!pub_done) publish();
        if (it >= 1 && !mbar_wait(ce, (it - 1) & 1)) *abort_flag = 1;
        if (!aborted(abort_flag)) {
          mbar_expect_tx(cf, (uint32_t)NP * CPB);
          const uint16_t* src = U.Cu + (long long)kk * U.cu_blk;
#pragma unroll
          for (int pp = 0; pp < NP; ++pp) bulk_g2s(sa(Cs) + pp * CPB, src + (long long)pp * 64 * KP, CPB, cf);
          ++ca;
        }
      }
      __syncwarp();
      for (int i0 = 0; i0 < nbt && !aborted(abort_flag); i0 += 32) {
        long long vo = 0, dofs = 0;
        if (i0 + lane < nbt) {
          const int p = X.blist[b0 + i0 + lane];
          vo = U.t1_idx[p] * U.vu_blk;
          const int di = P.v_didx[p];
          dofs = di >= 0 ? (long long)di * 256 : -1;   // a kept triplet always has its D block
        }
        const int nb = min(32, nbt - i0);
        for (int j = 0; j < nb; ++j) {
          const long long voj = __shfl_sync(0xffffffffu, vo, j);
          const long long doj = __shfl_sync(0xffffffffu, dofs, j);
          if (lane == 0 && doj < 0) *abort_flag = 1;
          if (lane == 0 && !aborted(abort_flag)) {
            const int s = db & 1;
            bool ok = db < 2 || mbar_wait(de + 8 * s, ((db >> 1) - 1) & 1);
            if (ok) {
              mbar_expect_tx(df + 8 * s, 1024u);
              bulk_g2s(sa(Ds + s * 256), U.Df + doj, 1024u, df + 8 * s);
              ++db;
            }
            ok = ok && (vb < 1 || mbar_wait(ve, (vb - 1) & 1));
            if (ok) {
              mbar_expect_tx(vf, (uint32_t)NP * 8192u);
              const uint16_t* src = U.Vu + voj;
#pragma unroll
              for (int pp = 0; pp < NP; ++pp) bulk_g2s(sa(Vs) + pp * 8192, src + pp * 4096, 8192u, vf);
              ++vb;
            } else {
              *abort_flag = 1;
            }
          }
          __syncwarp();
        }
      }
    }
    if (lane == 0) {
      if (ca) mbar_wait(cf, (ca - 1) & 1);
      if (vb) mbar_wait(vf, (vb - 1) & 1);
      for (int s = 0; s < 2; ++s) {
        const uint32_t n = db / 2 + ((uint32_t)s < db % 2 ? 1u : 0u);
        if (n) mbar_wait(df + 8 * s, (n - 1) & 1);
      }
    }
  } else if (warp == kWarpM) {
    // ------------------------------------------------------------ R issuer
    // R_B = C_AF . U_B^T (M = 64 alpha, N = beta, K = (f,a), one f per k
    // step) into one of two accumulators of kRCols columns.  A U piece
    // plane is 64 rows, i.e. eight 8-row groups, after the previous one, so
    // pieces 0 and 1 together are one N = 128 operand: block 0 (columns
    // 0-63) collects the products with U_0 (and U_2), block 1 those with U_1,
    // and R = block 0 + block 1.  BF16X6: C0 [U0;U1], C0 U2, C1 [U0;U1]
    // (C1 U1 comes with it), C2 U0; BF16X3: C0 [U0;U1], C1 U0.  Descriptors
    // are formed once; a k step adds 16 (256 bytes).
    constexpr int NR = NP == 3 ? 4 : 2;   // MMAs per k step
    const uint32_t idR128 = idesc_bf16(64, 128, 0), idR64 = idesc_bf16(64, 64, 0);
    const uint32_t rowg = 16u * KP;   // bytes between 8-row groups of C and U
    const uint64_t dC = sdesc2(sa(Cs), 128, rowg), dUR = sdesc2(sa(Us), 128, rowg);
    uint64_t pa[NR], pb[NR];
    uint32_t pid[NR];
    {
      const int ca[4] = {0, 0, 1, 2}, ub[4] = {0, 2, 0, 0}, wide[4] = {1, 0, 1, 0};   // BF16X6
      const int ca2[2] = {0, 1}, ub2[2] = {0, 0}, wide2[2] = {1, 0};                  // BF16X3
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        const int c = NP == 3 ? ca[k] : ca2[k], u = NP == 3 ? ub[k] : ub2[k], w = NP == 3 ? wide[k] : wide2[k];
        pa[k] = dC + ((uint64_t)(c * CPB) >> 4);
        pb[k] = dUR + ((uint64_t)(u * CPB) >> 4);
        pid[k] = w ? idR128 : idR64;
      }
    }
    uint32_t rb = 0, it = 0, ik = 0;
    bool ok = true;
    for (int kk = next_item(ik); kk < n_list; kk = next_item(ik), ++it) {
      const int q = qlist[kk];
      const int nbt = X.qcnt[q];
      if (lane == 0 && ok) {
        ok = mbar_wait(cf, it & 1);
        tc_fence_after();
        for (int i = 0; i < nbt && ok; ++i) {
          if (aborted(abort_flag)) {
            ok = false;
            break;
          }
          const int rbuf = rb & 1;
          const uint32_t dR = T + kRCol + (uint32_t)kRCols * rbuf;
          if (rb >= 2) ok = mbar_wait(re + 8 * rbuf, ((rb >> 1) - 1) & 1);
          for (int c = 0; c < 2 && ok; ++c) {
            ok = mbar_wait(uf + 8 * c, rb & 1);
            if (!ok) break;
            tc_fence_after();
            const int f0 = c ? FH : 0, f1 = c ? NF : FH;
            for (int f = f0; f < f1; ++f) {
              const uint64_t o = 16u * (uint32_t)f;
#pragma unroll
              for (int k = 0; k < NR; ++k) umma_bf16(dR, pa[k] + o, pb[k] + o, pid[k], (f > 0 || k > 0) ? 1u : 0u);
            }
            umma_commit(ue + 8 * c);
            if (c == 1) umma_commit(rf + 8 * rbuf);
          }
          ++rb;
        }
        if (ok) umma_commit(ce);
        if (!ok) *abort_flag = 1;
      }
      __syncwarp();
    }
  } else if (warp == kWarpQ) {
    // ------------------------------------------------------------ Q issuer
    // Q[:, chunk] += V_AB . U_B[:, chunk] (M = 64 alpha, N = the chunk's
    // (f,a) columns, K = beta in four k steps; U read MN-major).
    const int N0 = 16 * FH, N1 = 16 * (NF - FH);
    const uint32_t idQ0 = idesc_bf16(64, N0, 1), idQ1 = N1 > 0 ? idesc_bf16(64, N1, 1) : 0u;
    const uint32_t rowg = 16u * KP;
    const uint64_t dV = sdesc2(sa(Vs), 128, 1024), dUQ = sdesc2(sa(Us), rowg, 128);
    uint64_t pa[NPROD], pb[NPROD];
    {
      int k = 0;
#pragma unroll
      for (int sum = NP - 1; sum >= 0; --sum)
#pragma unroll
        for (int ia = 0; ia <= sum; ++ia, ++k) {
          pa[k] = dV + ((uint64_t)(ia * 8192) >> 4);
          pb[k] = dUQ + ((uint64_t)((sum - ia) * CPB) >> 4);
        }
    }
    const uint64_t kbA = 256 >> 4, kbB = (uint64_t)(2 * rowg) >> 4;
    uint32_t rb = 0, seg = 0, ik = 0;
    bool ok = true;
    for (int kk = next_item(ik); kk < n_list; kk = next_item(ik)) {
      const int q = qlist[kk];
      const int nbt = X.qcnt[q];
      if (lane == 0 && ok) {
        for (int i = 0; i < nbt && ok; ++i) {
          if (aborted(abort_flag)) {
            ok = false;
            break;
          }
          const bool first = (i % SEG) == 0, last = (i % SEG) == SEG - 1 || i == nbt - 1;
          for (int c = 0; c < 2 && ok; ++c) {
            ok = mbar_wait(uf + 8 * c, rb & 1);
            if (ok && c == 0) ok = mbar_wait(vf, rb & 1) && (!first || seg == 0 || mbar_wait(qe, (seg - 1) & 1));
            if (!ok) break;
            tc_fence_after();
            const int f0 = c ? FH : 0;
            const int Nc = c ? N1 : N0;
            if (Nc > 0) {
              const uint32_t idQ = c ? idQ1 : idQ0, tq = T + 16u * f0;
              const uint64_t oB = (uint64_t)(f0 * 256) >> 4;
              for (int kb = 0; kb < 4; ++kb)
#pragma unroll
                for (int k = 0; k < NPROD; ++k)
                  umma_bf16(tq, pa[k] + kbA * kb, pb[k] + oB + kbB * kb, idQ, (first && kb == 0 && k == 0) ? 0u : 1u);
            }
            umma_commit(ue + 8 * c);
          }
          if (!ok) break;
          umma_commit(ve);
          if (last) {
            umma_commit(qf);
            ++seg;
          }
          ++rb;
        }
        if (!ok) *abort_flag = 1;
      }
      __syncwarp();
    }
  } else if (warp >= kWarpE && warp < kWarpE + kNE) {
    // --------------------------------------------------------------- epilogue
    const int qd = warp & 3;                 // tensor-memory lane quarter
    const int ew = warp - kWarpE;
    const int alpha = qd * 16 + (lane & 15); // accumulator row held by this thread
    const int half = lane >> 4;              // columns [0,16) or [16,32) of a 32-column load
    const uint32_t tl = T + ((uint32_t)(qd * 32) << 16);
    uint32_t rb = 0, seg = 0, it = 0, ik = 0;
    double fl = 0.0;
    bool ok = true;
    for (int kk = next_item(ik); kk < n_list && ok; kk = next_item(ik), ++it) {
      const int q = qlist[kk];
      const int A = P.c_home[q], F = P.c_j[q];
      const int sA = P.species[A];
      const int nA = P.n_ao[sA], mA = P.n_abf[sA], nF = P.n_ao[P.species[F]];
      const long long b0 = X.qoff[q];
      const int nbt = X.qcnt[q];
      const float* Cf = reinterpret_cast<const float*>(U.Cu + (long long)kk * U.cu_blk + (long long)NP * 64 * KP);
      double e_it = 0.0, g_it[3] = {0.0, 0.0, 0.0};
      for (int i0 = 0; i0 < nbt && ok; i0 += 32) {
        int p_l = 0, mB_l = 0, nB_l = 0;
        long long vo_l = 0;
        if (i0 + lane < nbt) {
          p_l = X.blist[b0 + i0 + lane];
          const int sb = P.species[P.v_j[p_l]];
          mB_l = P.n_abf[sb];
          nB_l = P.n_ao[sb];
          vo_l = U.t1_idx[p_l] * U.vu_blk;
        }
        const int nb = min(32, nbt - i0);
        for (int j = 0; j < nb && ok; ++j) {
          ok = __all_sync(0xffffffffu, !aborted(abort_flag)) != 0;
          if (!ok) break;
          const int i = i0 + j;
          const int p = __shfl_sync(0xffffffffu, p_l, j);
          const int mB = __shfl_sync(0xffffffffu, mB_l, j);
          const int nB = __shfl_sync(0xffffffffu, nB_l, j);
          const long long vo = __shfl_sync(0xffffffffu, vo_l, j);
          const float* dV = reinterpret_cast<const float*>(U.Vu + vo + NP * 4096);
          const bool last = (i % SEG) == SEG - 1 || i == nbt - 1;
          const int rbuf = rb & 1;
          // ---- R_B -> g^V_AB (the grad V rows of the first 32 columns are
          // fetched before the wait; they do not depend on R)
          float gv[3] = {0.f, 0.f, 0.f};
          float4 w[3][4];
          const float4* dV4 = reinterpret_cast<const float4*>(dV) + qd * 32 + lane;   // epilogue load order (ep_at)
          {
            const int cb = 16 * half;
            if (alpha < mA && cb < mB)
#pragma unroll
              for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int t4 = 0; t4 < 4; ++t4) w[c][t4] = dV4[c * 1024 + t4 * 128];
          }
          ok = wait_all(rf + 8 * rbuf, (rb >> 1) & 1);
          tc_fence_after();
          if (ok) {
            for (int c0 = 0; c0 < 64; c0 += 32) {
              if (c0 >= mB) break;
              const int cb = c0 + 16 * half;
              const bool act = alpha < mA && cb < mB;
              if (c0 > 0 && act)
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                  for (int t4 = 0; t4 < 4; ++t4) w[c][t4] = dV4[c * 1024 + 512 + t4 * 128];
              // R = block 0 + block 1: each block dotted in turn (the dots are linear in R)
#pragma unroll 1
              for (int blk = 0; blk < 2; ++blk) {
                uint32_t v[32];
                tmem_ld32(tl + kRCol + (uint32_t)kRCols * rbuf + 64u * blk + c0, v);
                float x[16];
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                  const float hi = __shfl_sync(0xffffffffu, __uint_as_float(v[16 + t]), lane & 15);
                  x[t] = half ? hi : __uint_as_float(v[t]);
                }
                if (act) {
#pragma unroll
                  for (int c = 0; c < 3; ++c) {
                    float s = 0.f;
#pragma unroll
                    for (int t4 = 0; t4 < 4; ++t4) {
                      s = fmaf(w[c][t4].x, x[4 * t4], s);
                      s = fmaf(w[c][t4].y, x[4 * t4 + 1], s);
                      s = fmaf(w[c][t4].z, x[4 * t4 + 2], s);
                      s = fmaf(w[c][t4].w, x[4 * t4 + 3], s);
                    }
                    gv[c] += s;
                  }
                }
              }
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(re + 8 * rbuf);
#pragma unroll
          for (int c = 0; c < 3; ++c) gv[c] = warp_sum_f(gv[c]);
          if (lane == 0 && ok)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              if (gv[c] != 0.f) dev::add_gV(P, 3 * p + c, -(double)gv[c]);
          if (ew == 0 && lane == 0) fl += 2.0 * mB * nA * nB * nF + 4.0 * mA * mB * nA * nF;
          ++rb;
          // ---- end of a run: Q -> E, g^C
          if (last && ok) {
            ok = wait_all(qf, seg & 1);
            tc_fence_after();
            if (ok) {
              for (int c0 = 0; c0 < KP; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tl + c0, v);
                float x[16];
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                  const float hi = __shfl_sync(0xffffffffu, __uint_as_float(v[16 + t]), lane & 15);
                  x[t] = half ? hi : __uint_as_float(v[t]);
                }
                const int cb = c0 + 16 * half;
                if (alpha < mA && cb < KP) {
                  float s4[4];
#pragma unroll
                  for (int c = 0; c < 4; ++c) {
                    const float4* src =
                        reinterpret_cast<const float4*>(Cf + (long long)c * 64 * KP32) + (c0 >> 5) * 512 + qd * 32 + lane;
                    float s = 0.f;
#pragma unroll
                    for (int t4 = 0; t4 < 4; ++t4) {
                      const float4 w = src[t4 * 128];
                      s = fmaf(w.x, x[4 * t4], s);
                      s = fmaf(w.y, x[4 * t4 + 1], s);
                      s = fmaf(w.z, x[4 * t4 + 2], s);
                      s = fmaf(w.w, x[4 * t4 + 3], s);
                    }
                    s4[c] = s;
                  }
                  e_it += (double)s4[0];
                  g_it[0] += (double)s4[1];
                  g_it[1] += (double)s4[2];
                  g_it[2] += (double)s4[3];
                }
              }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(qe);
            ++seg;
          }
        }
      }
      // item totals: E and g^C_AF
      e_it = warp_sum_d(e_it);
#pragma unroll
      for (int c = 0; c < 3; ++c) g_it[c] = warp_sum_d(g_it[c]);
      if (lane == 0 && ok) {
        if (e_it != 0.0) dev::add_E(P, -e_it);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (g_it[c] != 0.0) dev::add_gC(P, 3 * q + c, -2.0 * g_it[c]);
      }
    }
    if (!ok) *abort_flag = 1;
    if (ew == 0 && lane == 0 && fl != 0.0) atomicAdd(&P.acc[ACC_F1], fl);
  } else if (warp >= kWarpU) {
    // ---------------------------------------------------------------------- U
    // Lane l of U warp uw: row beta = 8 uw + ((l >> 1) & 7), columns
    // a = 4 qa .. 4 qa + 3 with qa = 2 (l >> 4) + (l & 1).  A half warp then
    // stores one contiguous 128-byte run of U, and the four lanes of a row
    // read the same Y row (one shared-memory wavefront per 16-byte chunk for
    // the warp's eight rows).
    const int uw = warp - kWarpU;
    const int r8 = (lane >> 1) & 7, qa = 2 * (lane >> 4) + (lane & 1);
    const int beta = 8 * uw + r8;
    const int ysw = 2 * ((beta >> 1) & 1);          // chunk c of row beta is stored at c ^ ysw
    uint16_t* urow = Us + (beta >> 3) * KP * 8 + (beta & 7) * 8 + (qa & 1) * 4;
    uint32_t ub = 0, ys = 0, ik = 0;
    bool ok = true;
    for (int kk = next_item(ik); kk < n_list && ok; kk = next_item(ik)) {
      const int q = qlist[kk];
      const int nF = P.n_ao[P.species[P.c_j[q]]];
      const long long b0 = X.qoff[q];
      const int nbt = X.qcnt[q];
      for (int i0 = 0; i0 < nbt && ok; i0 += 32) {
        int mB_l = 0;
        if (i0 + lane < nbt) mB_l = P.n_abf[P.species[P.v_j[X.blist[b0 + i0 + lane]]]];
        const int nb = min(32, nbt - i0);
        for (int j = 0; j < nb && ok; ++j) {
          ok = __all_sync(0xffffffffu, !aborted(abort_flag)) != 0;
          if (!ok) break;
          const int mB = __shfl_sync(0xffffffffu, mB_l, j);
          const int s = ub & 1;
          ok = wait_all(df + 8 * s, (ub >> 1) & 1);
          if (!ok) break;
          float2 dd[2][16];   // (D_AB[4 qa + 2 j][b], D_AB[4 qa + 2 j + 1][b])
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
              const float4 w = *reinterpret_cast<const float4*>(Ds + s * 256 + (4 * qa + i) * 16 + 4 * (c4 ^ qa));
              float* col = (i & 1) ? &dd[i >> 1][0].y : &dd[i >> 1][0].x;
              col[2 * (4 * c4)] = w.x;
              col[2 * (4 * c4 + 1)] = w.y;
              col[2 * (4 * c4 + 2)] = w.z;
              col[2 * (4 * c4 + 3)] = w.w;
            }
          __syncwarp();
          if (lane == 0) mbar_arrive(de + 8 * s);
          for (int c = 0; c < 2 && ok; ++c) {
            if (ub >= 1) ok = wait_all(ue + 8 * c, (ub - 1) & 1);
            if (!ok) break;
            const int f0 = c ? FH : 0, f1 = c ? NF : FH;
            const int e = min(f1, nF);
            // rows f < nF, one Y slot per run [fa, fb); two f per pass (eight
            // independent FMA chains per lane)
            for (int fa = f0; fa < e && ok; fa += FS) {
              const int fb = min(fa + FS, e);
              const int sl = (int)(ys % NS);
              ok = wait_all(yf + 8 * sl, (ys / NS) & 1);
              if (!ok) break;
              if (NP == 3) {
                // BF16X6 (tighter on registers): one row per pass, each lane
                // reads the row's four 16-byte chunks (chunk c stored at c ^ ysw)
                for (int f = fa; f < fb; ++f) {
                  float y[16];
#pragma unroll
                  for (int c4 = 0; c4 < 4; ++c4) {
                    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (beta < mB)
                      a = *reinterpret_cast<const float4*>(Ys + sl * SLOT + ((f - fa) * mB + beta) * 16 + 4 * (c4 ^ ysw));
                    y[4 * c4] = a.x;
                    y[4 * c4 + 1] = a.y;
                    y[4 * c4 + 2] = a.z;
                    y[4 * c4 + 3] = a.w;
                  }
                  float uf4[4] = {0.f, 0.f, 0.f, 0.f};
                  if (beta < mB)
#pragma unroll
                    for (int b = 0; b < 16; ++b)
#pragma unroll
                      for (int j = 0; j < 2; ++j) {
                        uf4[2 * j] = fmaf(y[b], dd[j][b].x, uf4[2 * j]);
                        uf4[2 * j + 1] = fmaf(y[b], dd[j][b].y, uf4[2 * j + 1]);
                      }
                  if (f + 1 >= fb) {   // the slot's rows have been read and used
                    __syncwarp();
                    if (lane == 0) mbar_arrive(ye + 8 * sl);
                  }
                  uint2 pk[NP];
                  split4<NP>(uf4, pk);
#pragma unroll
                  for (int pp = 0; pp < NP; ++pp)
                    *reinterpret_cast<uint2*>(urow + (size_t)pp * 64 * KP + (2 * f + (qa >> 1)) * 64) = pk[pp];
                }
              } else {
                // BF16X3: the run's rows rho = (f - fa) mB + beta (the slot's
                // own order) are shared by all U warps, two per lane and pass
                // (rho = 16 g + r8 and 16 g + 8 + r8 for row groups g = uw,
                // uw + kNU, ...), so every warp gets the same share whatever
                // n_abf(B) is; rows beta >= n_abf(B) are zeroed after the chunk
                const int nrows = (fb - fa) * mB;
                const float* ysl = Ys + sl * SLOT;
                const float inv = 1.0f / (float)mB;
                for (int g = uw; 16 * g < nrows; g += kNU) {
                  int rho[2], fr[2], be[2];
                  rho[0] = 16 * g + r8;
                  rho[1] = rho[0] + 8;
#pragma unroll
                  for (int h = 0; h < 2; ++h) {   // (f - fa, beta) of row rho, exact after the correction
                    int t = (int)((float)rho[h] * inv);
                    if (t * mB > rho[h]) --t;
                    else if ((t + 1) * mB <= rho[h]) ++t;
                    fr[h] = t;
                    be[h] = rho[h] - t * mB;
                  }
                  const bool v0 = rho[0] < nrows, v1 = rho[1] < nrows;
                  // the two Y rows of this lane (16-byte chunk c stored at c ^ 2 ((beta >> 1) & 1))
                  float y0[16], y1[16];
  #pragma unroll
                  for (int c4 = 0; c4 < 4; ++c4) {
                    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
                    if (v0) a0 = *reinterpret_cast<const float4*>(ysl + rho[0] * 16 + 4 * (c4 ^ (2 * ((be[0] >> 1) & 1))));
                    if (v1) a1 = *reinterpret_cast<const float4*>(ysl + rho[1] * 16 + 4 * (c4 ^ (2 * ((be[1] >> 1) & 1))));
                    y0[4 * c4] = a0.x;
                    y0[4 * c4 + 1] = a0.y;
                    y0[4 * c4 + 2] = a0.z;
                    y0[4 * c4 + 3] = a0.w;
                    y1[4 * c4] = a1.x;
                    y1[4 * c4 + 1] = a1.y;
                    y1[4 * c4 + 2] = a1.z;
                    y1[4 * c4 + 3] = a1.w;
                  }
                  // u[a] = sum_b y[b] D[a][b] for four a of each row
                  float2 u0[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, u1[2] = {u0[0], u0[1]};
  #pragma unroll
                  for (int b = 0; b < 16; ++b)
  #pragma unroll
                    for (int j = 0; j < 2; ++j) {
                      u0[j].x = fmaf(y0[b], dd[j][b].x, u0[j].x);
                      u0[j].y = fmaf(y0[b], dd[j][b].y, u0[j].y);
                      u1[j].x = fmaf(y1[b], dd[j][b].x, u1[j].x);
                      u1[j].y = fmaf(y1[b], dd[j][b].y, u1[j].y);
                    }
                  uint2 pk[NP];
                  if (v0) {
                    float uf4[4] = {u0[0].x, u0[0].y, u0[1].x, u0[1].y};
                    split4<NP>(uf4, pk);
                    uint16_t* ur = Us + (be[0] >> 3) * KP * 8 + (be[0] & 7) * 8 + (qa & 1) * 4 +
                                   (2 * (fa + fr[0]) + (qa >> 1)) * 64;
  #pragma unroll
                    for (int pp = 0; pp < NP; ++pp) *reinterpret_cast<uint2*>(ur + (size_t)pp * 64 * KP) = pk[pp];
                  }
                  if (v1) {
                    float ug4[4] = {u1[0].x, u1[0].y, u1[1].x, u1[1].y};
                    split4<NP>(ug4, pk);
                    uint16_t* ur = Us + (be[1] >> 3) * KP * 8 + (be[1] & 7) * 8 + (qa & 1) * 4 +
                                   (2 * (fa + fr[1]) + (qa >> 1)) * 64;
  #pragma unroll
                    for (int pp = 0; pp < NP; ++pp) *reinterpret_cast<uint2*>(ur + (size_t)pp * 64 * KP) = pk[pp];
                  }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(ye + 8 * sl);   // every row of the slot has been read
              }
              ++ys;
            }
            // rows beta >= n_abf(B) (BF16X3 computes only the rows it reads)
            // and rows f >= nF of the chunk are zero
            if (NP == 2 && beta >= mB)
              for (int f = f0; f < e; ++f)
#pragma unroll
                for (int pp = 0; pp < NP; ++pp)
                  *reinterpret_cast<uint2*>(urow + (size_t)pp * 64 * KP + (2 * f + (qa >> 1)) * 64) = make_uint2(0u, 0u);
            for (int f = max(f0, e); f < f1; ++f)
#pragma unroll
              for (int pp = 0; pp < NP; ++pp)
                *reinterpret_cast<uint2*>(urow + (size_t)pp * 64 * KP + (2 * f + (qa >> 1)) * 64) = make_uint2(0u, 0u);
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(uf + 8 * c);
          }
          ++ub;
        }
      }
    }
    if (!ok) *abort_flag = 1;
  }
  // ------------------------------------------------------------------ teardown
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kWarpM) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(T), "r"(512));
  if (tid == 0 && s_abort) atomicExch(err, 1);
}

// ------------------------------------------------------------------ R2 and Z
// Second exchange product on the tensor cores, per kept pair (A,B) of the
// pass (slot kk of its list), shapes n_abf <= 64, n_ao <= 16:
//   R2 = Y^{AB} . (Y^{BA})^T (M = 64 alpha, N = 64 beta, K = (a, b)) -> E = -<V, R2>, g^V = -<grad V, R2>
//   Z  = V_AB . Y^{BA}       (M = 64 alpha, N = (a, b), K = beta)    -> the Z store read by k_q2_umma
// Both Y operands come whole from the Y build's core-matrix stores (X.ycm):
// Y^{AB} from YspT (rows alpha, K = (a, b)), Y^{BA} from Ysp (rows beta,
// K = (a, b)); Y^{BA} serves R2 as a K-major and Z as an MN-major operand.
// V pieces and FP32 V, grad V from X.Vz.  CTA c takes the pairs c, c + grid,
// ...  Warp 0 lane 0 copies (bulk), warp 1 owns tensor memory and its lane 0
// issues the MMAs, warps 2-5 (one per tensor-memory lane quarter) are the
// epilogue.  R2 is double-buffered in tensor memory, Z single-buffered;
// Y^{AB} is released after R2, Y^{BA} and V after Z, so the next pair's
// Y^{AB} lands while Z runs.  Every wait is bounded (1 s); a timeout sets the
// error flag and every role stops.
constexpr int kT2Threads = 192;
constexpr int kT2RCol = 256;   // tensor-memory column of the first R2 accumulator (Z at column 0)

template <int NP>
__global__ void __launch_bounds__(kT2Threads, 1)
    k_t2_umma(DevPlan P, MixPlan X, const int* list, int n_list, int KKmax, long long zblk, int* err) {
  constexpr int NPROD = NP * (NP + 1) / 2;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint16_t* Ya = reinterpret_cast<uint16_t*>(smem_raw);   // [NP][64][KK]
  uint16_t* Yb = Ya + (size_t)NP * 64 * KKmax;            // [NP][64][KK]
  uint16_t* Vs = Yb + (size_t)NP * 64 * KKmax;            // [NP][64][64]
  __shared__ __align__(8) uint64_t b_af, b_ae, b_bf, b_be, b_rf[2], b_re[2], b_zf, b_ze, b_done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  volatile int* abort_flag = &s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto sa = [](const void* p) { return (uint32_t)__cvta_generic_to_shared(p); };
  const uint32_t mAf = sa(&b_af), mAe = sa(&b_ae), mBf = sa(&b_bf), mBe = sa(&b_be), rf = sa(b_rf), re = sa(b_re),
                 zf = sa(&b_zf), ze = sa(&b_ze), mdone = sa(&b_done);
  if (tid == 0) {
    s_abort = 0;
    mbar_init(mAf, 1);
    mbar_init(mAe, 1);
    mbar_init(mBf, 1);
    mbar_init(mBe, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(rf + 8 * s, 1);
      mbar_init(re + 8 * s, 4);
    }
    mbar_init(zf, 1);
    mbar_init(ze, 4);
    mbar_init(mdone, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sa(&tmem_base)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t T = tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------- producer
    if (lane == 0) {
      uint32_t na = 0, nb = 0;   // copies issued into Ya and into Yb / V
      for (int kk = blockIdx.x; kk < n_list && !aborted(abort_flag); kk += gridDim.x) {
        const int p = list[kk];
        const int A = P.v_home[p], b = P.v_j[p];
        const int* Rb = P.v_R + 3 * p;
        const int KK = 16 * P.n_ao[P.species[A]];
        const int y1 = ylut_get(P, A, b, Rb[0], Rb[1], Rb[2]);
        const int y2 = ylut_get(P, b, A, -Rb[0], -Rb[1], -Rb[2]);
        if (y1 < 0 || y2 < 0) {   // a kept pair always has both Y blocks
          *abort_flag = 1;
          break;
        }
        const uint32_t ybytes = (uint32_t)NP * 64u * (uint32_t)KK * 2u;
        if (na >= 1 && !mbar_wait(mAe, (na - 1) & 1)) {
          *abort_flag = 1;
          break;
        }
        mbar_expect_tx(mAf, ybytes);
        bulk_g2s(sa(Ya), X.YspT + X.y_idx[y1] * X.yT_blk, ybytes, mAf);
        ++na;
        if (nb >= 1 && !mbar_wait(mBe, (nb - 1) & 1)) {
          *abort_flag = 1;
          break;
        }
        mbar_expect_tx(mBf, ybytes + (uint32_t)NP * 8192u);
        bulk_g2s(sa(Yb), X.Ysp + P.y_off[y2], ybytes, mBf);
        bulk_g2s(sa(Vs), X.Vz + (long long)kk * X.vz_blk, (uint32_t)NP * 8192u, mBf);
        ++nb;
      }
      // copies in flight land before the CTA leaves
      if (na) mbar_wait(mAf, (na - 1) & 1);
      if (nb) mbar_wait(mBf, (nb - 1) & 1);
    }
  } else if (warp == 1) {
    // ----------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idR = idesc_bf16(64, 64, 0);
      uint32_t i = 0;
      bool ok = true;
      for (int kk = blockIdx.x; kk < n_list && ok; kk += gridDim.x, ++i) {
        if (aborted(abort_flag)) {
          ok = false;
          break;
        }
        const int nA = P.n_ao[P.species[P.v_home[list[kk]]]];
        const int KK = 16 * nA;
        const uint32_t PB = 64u * (uint32_t)KK * 2u;   // bytes of one piece of Y^{AB} or Y^{BA}
        const uint32_t rowg = 16u * (uint32_t)KK;      // bytes between 8-row groups
        const uint64_t dA = sdesc2(sa(Ya), 128, rowg), dBK = sdesc2(sa(Yb), 128, rowg);
        const uint64_t dV = sdesc2(sa(Vs), 128, 1024), dBM = sdesc2(sa(Yb), rowg, 128);
        const uint32_t idZ = idesc_bf16(64, KK, 1);
        const int rbuf = i & 1;
        ok = mbar_wait(mAf, i & 1) && mbar_wait(mBf, i & 1) && (i < 2 || mbar_wait(re + 8 * rbuf, ((i >> 1) - 1) & 1));
        if (!ok) break;
        tc_fence_after();
        // R2: one a (16 columns, 256 bytes) per k step, every piece product
        const uint32_t tR = T + kT2RCol + 64u * rbuf;
        for (int a = 0; a < nA; ++a) {
          const uint64_t o = 16u * (uint32_t)a;
          int k = 0;
#pragma unroll
          for (int sum = NP - 1; sum >= 0; --sum)
#pragma unroll
            for (int ia = 0; ia <= sum; ++ia, ++k)
              umma_bf16(tR, dA + ((uint64_t)(ia * PB) >> 4) + o, dBK + ((uint64_t)((sum - ia) * PB) >> 4) + o, idR,
                        (a > 0 || k > 0) ? 1u : 0u);
        }
        umma_commit(mAe);
        umma_commit(rf + 8 * rbuf);
        ok = i < 1 || mbar_wait(ze, (i - 1) & 1);
        if (!ok) break;
        tc_fence_after();
        // Z: K = beta in four steps of 16 (V: 256 bytes; Y^{BA} MN-major: two 8-row groups)
        for (int kb = 0; kb < 4; ++kb) {
          int k = 0;
#pragma unroll
          for (int sum = NP - 1; sum >= 0; --sum)
#pragma unroll
            for (int ia = 0; ia <= sum; ++ia, ++k)
              umma_bf16(T, dV + ((uint64_t)(ia * 8192) >> 4) + 16u * kb,
                        dBM + ((uint64_t)((sum - ia) * PB) >> 4) + ((uint64_t)(2 * rowg * kb) >> 4), idZ,
                        (kb > 0 || k > 0) ? 1u : 0u);
        }
        (void)NPROD;
        umma_commit(mBe);
        umma_commit(zf);
      }
      if (!ok) *abort_flag = 1;
      // every MMA issued has completed before tensor memory is freed
      umma_commit(mdone);
      mbar_wait(mdone, 0);
    }
  } else {
    // ------------------------------------------------------------- epilogue
    const int qd = warp & 3;                   // tensor-memory lane quarter
    const int alpha = qd * 16 + (lane & 15);   // accumulator row held by this thread
    const int half = lane >> 4;                // columns [0,16) or [16,32) of a 32-column load
    const uint32_t tl = T + ((uint32_t)(qd * 32) << 16);
    uint32_t i = 0;
    bool ok = true;
    double fl = 0.0;
    for (int kk = blockIdx.x; kk < n_list && ok; kk += gridDim.x, ++i) {
      ok = __all_sync(0xffffffffu, !aborted(abort_flag)) != 0;
      if (!ok) break;
      const int p = list[kk];
      const int sA = P.species[P.v_home[p]], sB = P.species[P.v_j[p]];
      const int nA = P.n_ao[sA], nB = P.n_ao[sB], mA = P.n_abf[sA], mB = P.n_abf[sB];
      const int KK = 16 * nA;
      const int rbuf = i & 1;
      // ---- R2 -> E, g^V (the V, grad V rows of the first 32 columns are
      // fetched before the wait; they do not depend on R2)
      const float4* V4 = reinterpret_cast<const float4*>(X.Vz + (long long)kk * X.vz_blk + NP * 4096) + qd * 32 + lane;
      float ev[4] = {0.f, 0.f, 0.f, 0.f};
      float4 w[4][4];
      if (alpha < mA && 16 * half < mB)
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int t4 = 0; t4 < 4; ++t4) w[c][t4] = V4[c * 1024 + t4 * 128];
      ok = wait_all(rf + 8 * rbuf, (i >> 1) & 1);
      tc_fence_after();
      if (ok) {
        for (int c0 = 0; c0 < 64; c0 += 32) {
          if (c0 >= mB) break;
          const bool act = alpha < mA && c0 + 16 * half < mB;
          if (c0 > 0 && act)
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
              for (int t4 = 0; t4 < 4; ++t4) w[c][t4] = V4[c * 1024 + 512 + t4 * 128];
          uint32_t v[32];
          tmem_ld32(tl + kT2RCol + 64u * rbuf + c0, v);
          float x[16];
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const float hi = __shfl_sync(0xffffffffu, __uint_as_float(v[16 + t]), lane & 15);
            x[t] = half ? hi : __uint_as_float(v[t]);
          }
          if (act) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              float s = 0.f;
#pragma unroll
              for (int t4 = 0; t4 < 4; ++t4) {
                s = fmaf(w[c][t4].x, x[4 * t4], s);
                s = fmaf(w[c][t4].y, x[4 * t4 + 1], s);
                s = fmaf(w[c][t4].z, x[4 * t4 + 2], s);
                s = fmaf(w[c][t4].w, x[4 * t4 + 3], s);
              }
              ev[c] += s;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(re + 8 * rbuf);
#pragma unroll
      for (int c = 0; c < 4; ++c) ev[c] = warp_sum_f(ev[c]);
      if (lane == 0 && ok) {
        if (ev[0] != 0.f) dev::add_E(P, -(double)ev[0]);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (ev[c + 1] != 0.f) dev::add_gV(P, 3 * p + c, -(double)ev[c + 1]);
      }
      // ---- Z -> the Z store: NP planes of 128-row tiles of rows (alpha, a),
      // 16 columns b each, in the core-matrix order of tix; a thread writes
      // the 16 b of one (alpha, a) as two 16-byte chunks per piece
      ok = ok && wait_all(zf, i & 1);
      tc_fence_after();
      if (ok) {
        uint16_t* Zo = X.Zst + (long long)kk * zblk;
        for (int c0 = 0; c0 < KK; c0 += 32) {
          uint32_t v[32];
          tmem_ld32(tl + c0, v);
          float x[16];
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const float hi = __shfl_sync(0xffffffffu, __uint_as_float(v[16 + t]), lane & 15);
            x[t] = half ? hi : __uint_as_float(v[t]);
          }
          const int a = (c0 >> 4) + half;
          if (alpha < mA && a < nA) {
            const int r = alpha * nA + a;
            uint16_t* d = Zo + (long long)(r >> 7) * NP * 2048 + (((r & 127) >> 3) << 7) + ((r & 7) << 3);
#pragma unroll
            for (int hb = 0; hb < 2; ++hb) {
              const float x0[4] = {x[8 * hb], x[8 * hb + 1], x[8 * hb + 2], x[8 * hb + 3]};
              const float x1[4] = {x[8 * hb + 4], x[8 * hb + 5], x[8 * hb + 6], x[8 * hb + 7]};
              uint2 p0[NP], p1[NP];
              split4<NP>(x0, p0);
              split4<NP>(x1, p1);
#pragma unroll
              for (int pp = 0; pp < NP; ++pp)
                *reinterpret_cast<uint4*>(d + pp * 2048 + 64 * hb) = make_uint4(p0[pp].x, p0[pp].y, p1[pp].x, p1[pp].y);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(ze);
      if (warp == 2 && lane == 0) fl += 4.0 * mA * mB * nA * nB;
    }
    if (!ok) *abort_flag = 1;
    if (warp == 2 && lane == 0 && fl != 0.0) atomicAdd(&P.acc[ACC_F2], fl);
  }
  // ------------------------------------------------------------------ teardown
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(T), "r"(512));
  if (tid == 0 && s_abort) atomicExch(err, 1);
}

int num_sms() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 152;
  }();
  return n;
}

}  // namespace

long long t1u_launch_count() { return g_t1u_launches; }

size_t t1u_smem(int np, int KP, int NS, int FS) {
  return (size_t)np * 64 * KP * 2 * 2 + (size_t)np * 8192 + 2 * 256 * 4 + (size_t)NS * FS * 1024 * 4;
}

int t1u_max_slots() { return kMaxNS; }

cudaError_t t1u_set_smem(int np) {
  return allow_max_dynamic_smem(np == 2 ? (const void*)k_t1_umma<2> : (const void*)k_t1_umma<3>);
}

cudaError_t launch_t1u_stores(const DevPlan& P, const T1UPlan& U, int np, const int* qlist, int nq, bool dstore,
                              cudaStream_t s) {
  if (nq > 0) {
    ++g_t1u_launches;
    static std::once_flag attr;
    std::call_once(attr, [] {
      cudaFuncSetAttribute(k_t1u_cstore<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCStoreSmem);
      cudaFuncSetAttribute(k_t1u_cstore<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCStoreSmem);
    });
    const int g = nq < 152 * 3 ? nq : 152 * 3;
    if (np == 2) k_t1u_cstore<2><<<g, 256, kCStoreSmem, s>>>(P, U, qlist, nq);
    else k_t1u_cstore<3><<<g, 256, kCStoreSmem, s>>>(P, U, qlist, nq);
  }
  if (dstore && P.n_d > 0) {
    ++g_t1u_launches;
    const long long g = P.n_d < 152 * 16 ? P.n_d : 152 * 16;
    k_t1u_dstore<<<(unsigned)g, 256, 0, s>>>(P, U.Df);
  }
  return cudaGetLastError();
}

cudaError_t launch_lpt_order(const int* key, int asc, const int* list, int n_max, const long long* n_dev, int* hist,
                             int* out, cudaStream_t s) {
  if (n_max <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(hist, 0, kLptBuckets * sizeof(int), s);
  if (e != cudaSuccess) return e;
  g_t1u_launches += 3;
  const int g = std::min((n_max + 255) / 256, 152 * 8);
  k_lpt_hist<<<g, 256, 0, s>>>(key, asc, list, n_dev, hist);
  k_lpt_scan<<<1, 1024, 0, s>>>(hist);
  k_lpt_scatter<<<g, 256, 0, s>>>(key, asc, list, n_dev, hist, out);
  return cudaGetLastError();
}

cudaError_t launch_vstores(const DevPlan& P, const MixPlan& X, const T1UPlan& U, int np, const int* list, int n,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ++g_t1u_launches;
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_vstores<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kVStoreSmem);
    cudaFuncSetAttribute(k_vstores<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kVStoreSmem);
  });
  const int g = n < 152 * 3 ? n : 152 * 3;
  if (np == 2) k_vstores<2><<<g, 256, kVStoreSmem, s>>>(P, X, U, list, n);
  else k_vstores<3><<<g, 256, kVStoreSmem, s>>>(P, X, U, list, n);
  return cudaGetLastError();
}

size_t t2u_smem(int np, int max_ao) { return (size_t)np * (2 * 64 * 16 * (size_t)max_ao * 2 + 8192); }

cudaError_t t2u_set_smem(int np) {
  return allow_max_dynamic_smem(np == 2 ? (const void*)k_t2_umma<2> : (const void*)k_t2_umma<3>);
}

cudaError_t launch_t2_umma(const DevPlan& P, const MixPlan& X, int np, const int* list, int n, long long zblk,
                           size_t smem, int* err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ++g_t1u_launches;
  const int grid = n < num_sms() ? n : num_sms();
  const int KKmax = (int)(smem / np - 8192) / (2 * 64 * 2);   // 16 x the largest n_ao
  if (np == 2) k_t2_umma<2><<<grid, kT2Threads, smem, s>>>(P, X, list, n, KKmax, zblk, err);
  else k_t2_umma<3><<<grid, kT2Threads, smem, s>>>(P, X, list, n, KKmax, zblk, err);
  return cudaGetLastError();
}

cudaError_t launch_t1_umma(const DevPlan& P, const MixPlan& X, const T1UPlan& U, int np, const int* qlist, int n,
                           size_t smem, int* work, int* err, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  ++g_t1u_launches;
  const int grid = n < num_sms() ? n : num_sms();
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (np == 2) k_t1_umma<2><<<grid, kThreads, smem, s>>>(P, X, U, qlist, n, work, err);
  else k_t1_umma<3><<<grid, kThreads, smem, s>>>(P, X, U, qlist, n, work, err);
  return cudaGetLastError();
}

}  // namespace hfx
