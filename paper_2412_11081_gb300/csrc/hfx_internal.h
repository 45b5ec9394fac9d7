// Internal declarations shared by the host planner (hfx_host.cpp) and the
// CUDA kernels (hfx_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace hfx {

constexpr int kMaxSpecies = 16;
constexpr int kMaxAO = 32;
constexpr int kMaxABF = 128;
constexpr int kMaxCPerAtom = 256;     // C-pair candidates per home atom (mask width)
constexpr int kMaskWords = kMaxCPerAtom / 32;

// Everything a kernel needs, passed by value.  All pointers are device
// pointers.  Pair p of a list is (home atom *_home[p] -> atom *_j[p], image
// *_R[3p..3p+2]); its vector is d = tau_j + R.L - tau_home.
struct DevPlan {
  int N, S;
  const int* species;
  const int* n_ao;
  const int* n_abf;
  const long long* G_off;      // [S*S] element offsets of G_st (and G'_st)
  const double* G;
  const double* Gp;            // anisotropic templates or nullptr
  const long long* M_off;
  const double* M;
  const double* Mnorm;         // [S*S] ||M_st||_F
  const double* Gmom;          // [S*S*3] sum G^2, sum G G', sum G'^2 of each template pair
  // FP32 copies of G, G' (nullptr without anisotropy) and M: the split path
  // evaluates its FP32 operand stores from them (FP32 products of the
  // rounded templates and the rounded per-pair scalars), since GB300's FP64
  // pipe would otherwise bound those store kernels
  const float* Gf;
  const float* Gpf;
  const float* Mf;
  double e[3];
  double RC, omega;
  double thC, thdC, thV, thdV, thD, thCS;
  int terms;
  int h0, h1;                  // home atoms A whose items are screened in: [h0, h1)

  const double* pos;           // [N*3] current positions
  const double* L;             // [9] current lattice (rows), device memory (written before each evaluation)

  // density matrix
  long long n_d;
  const double* Dval;
  const long long* Doff;
  const int* Didx;             // [n_d*5]
  double* Dkept;               // [n_d] ||D|| if kept by step 1, else 0
  const int* dlut;             // dense (i, j, R) -> block index or -1
  int HD0, HD1, HD2;

  // C-pair candidates
  int nC;
  const int* c_ptr;            // [N+1]
  const int* c_home;
  const int* c_j;
  const int* c_R;
  const long long* c_off;      // element offset of C_p in Cst (grad C_p at 3*c_off in dCst)
  double* Cst;
  double* dCst;
  double* c_norm;              // max(||C||, ||grad C||) if kept, else 0
  double* c_sc;                // [nC*8] scalars of C = G f + G' fa, grad C = G g + G' ga (split path)
  unsigned char* c_keep;

  // V-pair candidates
  int nV;
  const int* v_ptr;
  const int* v_home;
  const int* v_j;
  const int* v_R;
  const int* v_didx;           // D block of (home, j, R) or -1
  double* v_norm;              // max(||V||, ||grad V||) if kept, else 0
  double* v_hg;                // [nV*4] h(r) and g = h'(r) d / r of the pair's V = M h, grad V = M g
  unsigned char* v_keep;
  unsigned int* v_mask;        // [nV*kMaskWords] kept F (C-pair slots of home)
  unsigned char* v_t2;         // kept for the second exchange product
  int* v_flag;                 // V block needed this call
  long long* v_off;            // offset of (V, grad V) in Vst
  double* Vst;

  // Y^{XZ} candidates (X home, Z = (j, R))
  int nY;
  const int* y_ptr;
  const int* y_home;
  const int* y_j;
  const int* y_R;
  double* yhat;
  int* y_flag;
  long long* y_off;
  double* Yst;
  const int* ylut;
  int HY0, HY1, HY2;

  // accumulators
  double* gC;                  // [nC*3] dE/dd for C pairs
  double* gV;                  // [nV*3]
  double* acc;                 // [0] E, [1..9] virial sum g (x) d, [10] flops y, [11] t1, [12] t2
  unsigned long long* cnt;     // [0] c kept, [1] v kept, [2] d kept, [3] triplets
  // deterministic plans: exact fixed-point cells (hfx_accum.cuh) of gC, gV,
  // E and the virial (fxA: E, then the nine virial components) and F, in
  // place of the FP64 atomics; all nullptr otherwise
  unsigned long long* fxC;
  unsigned long long* fxV;
  unsigned long long* fxA;
  unsigned long long* fxF;
};

// Extra state of the split-precision path.
struct MixPlan {
  uint16_t* Dsp;               // D blocks as bf16 pieces, rup16(n_ao(I)) x rup16(n_ao(J)) per piece
  const long long* dsp_off;    // [n_d]
  uint16_t* Ysp;               // Y^{XZ} as bf16 pieces, [alpha][z][rup16(n_ao(X))] per piece
  uint16_t* Cm;                // per C pair: bf16 pieces of C, then grad C in FP32
  const long long* cm_off;     // [nC] offsets (uint16 units)
  uint16_t* Vm;                // per needed V pair: bf16 pieces of V, then V and grad V in FP32
  const long long* vm_off;     // [nV] offsets (uint16 units), from the per-call scan
  uint16_t* Zst;               // per pair of the second product: bf16 pieces of Z = V_AB . Y^{BA}
  int* qcnt;                   // [nC] kept B per (A,F)
  long long* qoff;             // [nC] offsets into blist
  int* blist;                  // V pairs (A,B) per (A,F), in V-pair order
  float* Yf = nullptr;         // Y^{XZ} in FP32 as [z][alpha][16], offsets y_off / np (tcgen05 term 1 only)
  uint16_t* YspT = nullptr;    // Y^{XZ} transposed, bf16 pieces [piece][(alpha,x)][16 z] (z padded), yT_blk per key
  long long yT_blk = 0;        // uint16 units per key of YspT (np x 128-row tiles x 16)
  const long long* y_idx = nullptr;   // key -> its position in the needed-key list (YspT block)
  int* ytab = nullptr;         // Y build: D block (256-element units) per (key group, C slot t, key i), or -1
  int ytab_stride = 0;         // ints per key group (8 * most C pairs of an atom)
  int* q2tab = nullptr;        // second product: D block per (group of 8 C slots, pair slot, i), or -1
  // Fault injection for the failure tests: 1 = the second product's producer
  // issues no copies, so its pipeline waits run out (HFX_ERR_TIMEOUT).
  int stall_q2 = 0;
  // tcgen05 R2 / Z kernel (k_t2_umma): with ycm the Y build writes Ysp and
  // YspT per key as NP planes of 64 rows alpha x K columns in the tensor
  // cores' core-matrix order (Ysp: K = (z, x), 16 n_ao(Z) columns; YspT:
  // K = (x, z), 16 n_ao(X) columns; rows past n_abf(X) are left as they are:
  // finite, never read into a kept result); Vz holds per second-product pair
  // slot NP pieces of V [alpha 64][beta 64] in core-matrix order, then V and
  // grad V as four FP32 planes of 64 x 64 in epilogue load order.
  int ycm = 0;
  uint16_t* Vz = nullptr;
  long long vz_blk = 0;
  const long long* t2_slot = nullptr;   // V pair -> its slot in the pass's second-product list
  // 128-row tiles per CTA of the tcgen05 Y build and Q2 GEMM (1 or 2; the
  // autotuner's choice): two tiles share each K step's D blocks, one tile
  // runs more stages and two accumulators
  int ybtpc = 2;
  int q2tpc = 2;
};

// Element (row, f < 16) of one component of grad C_AF (FP32) in the C operand
// store, rows (alpha, a) in 128-row tiles: within a tile, four 128 x 4 column
// groups, a row's four values contiguous, so that 32 consecutive rows read
// one column group as 512 consecutive bytes.  A component spans
// ceil(rows / 128) * 2048 floats.
__host__ __device__ inline int gc_off(int row, int f) {
  return ((((row >> 7) * 4 + (f >> 2)) * 128 + (row & 127)) << 2) + (f & 3);
}

// Operand stores of the tcgen05 first-product kernel (hfx_t1umma.cu).
struct T1UPlan {
  uint16_t* Cu;                // per item (A,F): np bf16 pieces of C as [alpha 64][(f,a) KP], then C, grad C FP32 [4][64][KP]
  long long cu_blk;            // uint16 units per item
  uint16_t* Vu;                // per term-1 V pair: np pieces of V [alpha 64][beta 64], then grad V FP32 [3][64][64]
  long long vu_blk;            // uint16 units per V pair
  const long long* t1_idx;     // V pair -> its position in the term-1 V list
  float* Yf;                   // see MixPlan::Yf
  float* Df;                   // D blocks in FP32, [16][16] each
  int KP;                      // columns (f,a) = 16 f + a: 16 * max n_ao
  int NS;                      // Y ring slots
  int FS;                      // rows f per Y slot (a run never crosses a U chunk)
  int seg;                     // B per FP32 run of the Q accumulator
};

enum AccSlot { ACC_E = 0, ACC_W = 1, ACC_FY = 10, ACC_F1 = 11, ACC_F2 = 12, ACC_N = 16 };
enum CntSlot { CNT_C = 0, CNT_V = 1, CNT_D = 2, CNT_TRIP = 3, CNT_N = 8 };

// Kernels launched by this library since load (every launcher adds its
// launches); the host reads it before and after a call.
long long launch_count();

// Kernel launchers (hfx_kernels.cu).  Each returns the launch's cudaError_t.
cudaError_t launch_dnorm(const DevPlan& P, cudaStream_t s);
cudaError_t launch_cblocks(const DevPlan& P, int frozen, cudaStream_t s);
// Split path: per-pair scalars of C and the step-1 decision from the
// template moments, without writing the FP64 blocks.
cudaError_t launch_cnorm(const DevPlan& P, int frozen, cudaStream_t s);
cudaError_t launch_vnorm(const DevPlan& P, int frozen, cudaStream_t s);
cudaError_t launch_yhat(const DevPlan& P, cudaStream_t s);
cudaError_t launch_screen(const DevPlan& P, cudaStream_t s);
cudaError_t launch_vblocks(const DevPlan& P, const int* v_list, int n, cudaStream_t s);
cudaError_t launch_ybuild(const DevPlan& P, const int* y_list, int n, cudaStream_t s);
cudaError_t launch_term1(const DevPlan& P, const int* list, int n, int beta_chunk, size_t smem,
                         cudaStream_t s);
cudaError_t launch_term2(const DevPlan& P, const int* list, int n, int alpha_chunk, size_t smem,
                         cudaStream_t s);
cudaError_t launch_reduce(const DevPlan& P, double* out, cudaStream_t s);
// Plans created and evaluated from different host threads share the
// kernels' attributes, so no plan sets a kernel's dynamic shared-memory cap
// to its own size: allow_max_dynamic_smem raises the cap of f to the
// device's opt-in maximum minus f's static shared memory, the same value
// from every caller (each plan checks its own sizes against that limit).
cudaError_t allow_max_dynamic_smem(const void* f);
cudaError_t set_kernel_smem_limits();
// Batched LRI fit (hfx_lri_fit): X = A^-1 B and dX[c] = A^-1 (dB[c] - dA[c] X)
// per pair, device pointers, dA / dB / dX null for X alone; *err = 1 when a
// metric is not positive definite.
size_t lri_fit_smem(int n);
cudaError_t launch_lri_fit(int batch, int n, int w, const double* A, const double* B, const double* dA,
                           const double* dB, double* X, double* dX, int* err, cudaStream_t s);

// Split-precision kernels (hfx_mixed.cu); np = bf16 pieces per operand (2 or 3).
long long mixed_launch_count();
cudaError_t launch_dsplit(const DevPlan& P, const MixPlan& X, int np, cudaStream_t s);
cudaError_t launch_cpieces(const DevPlan& P, const MixPlan& X, int np, cudaStream_t s);
cudaError_t launch_vpieces(const DevPlan& P, const MixPlan& X, int np, const int* list, int n, cudaStream_t s);
cudaError_t launch_ygroups(const DevPlan& P, const long long* y_idx, const long long* y_total, int* gcnt,
                           const long long* goff, int* gX, int* gS, int* gN, int phase, cudaStream_t s);
// The D piece store viewed as a 2-D tensor of 512-byte rows (one row per
// bf16 piece of a 16 x 16 block, row dsp_off / 256 + piece; the last row is
// zero), fetched four rows at a time by the tensor-core kernels.
struct DRows {
  CUtensorMap map;             // box: one row of 256 bf16
  int zero_row;
};
cudaError_t launch_ybuild_mma(const DevPlan& P, const MixPlan& X, int np, const int* ylist, const int* gX,
                              const int* gS, const int* gN, int ngroups, int MC, const DRows& drows, int* err,
                              cudaStream_t s);
// ints of the D-block tables (MixPlan::ytab, MixPlan::q2tab)
long long ytab_size(int ngroups, int maxC);
long long q2tab_size(int n_slots, int FC);
cudaError_t launch_t1_lists(const DevPlan& P, const MixPlan& X, int phase, cudaStream_t s);
size_t term1_mma_smem(int np, int MAmax, int MBmax, int KSmax, int YRmax);
size_t term2_mma_smem(int np, int MAmax, int KZmax);
cudaError_t set_mixed_smem_limits(int np);
cudaError_t launch_term1_mma(const DevPlan& P, const MixPlan& X, int np, const int* qlist, int n, int MAmax,
                             int MBmax, int KSmax, int YRmax, size_t smem, cudaStream_t s);
// Second product of the home atoms [a0, a1): list / slot0 / n are that pass's
// pair list, its slot of every V pair of those atoms and its length.
cudaError_t launch_term2_mma(const DevPlan& P, const MixPlan& X, int np, const int* list, const long long* slot0,
                             int n, int a0, int a1, int MAmax, int KZmax, long long zblk, int zrows, int FC, int MC,
                             int nseg, int flush, const DRows& drows, size_t smem, int* err, cudaStream_t s,
                             bool pairs_done = false);
int q2_umma_segments(int max_pairs_per_atom, int np, int tpc);
// R2 and Z of the pass's second-product pairs on tcgen05 (hfx_t1umma.cu),
// shapes n_abf <= 64, n_ao <= 16, with X.ycm and X.Vz set: E, g^V and the Z
// store that k_q2_umma reads (launch_term2_mma with pairs_done then skips
// its warp-level R2 / Z kernel).
size_t t2u_smem(int np, int max_ao);
cudaError_t t2u_set_smem(int np);
cudaError_t launch_t2_umma(const DevPlan& P, const MixPlan& X, int np, const int* list, int n, long long zblk,
                           size_t smem, int* err, cudaStream_t s);

// tcgen05 first exchange product (hfx_t1umma.cu): shapes n_abf <= 64, n_ao <= 16.
long long t1u_launch_count();
size_t t1u_smem(int np, int KP, int NS, int FS);
// Columns of one FP32 plane of C / grad C in the operand store (KP rounded up to 32).
__host__ __device__ inline int t1u_kp32(int KP) { return (KP + 31) & ~31; }
// Items of the first product in a chosen order: list[0..*n) (n read on the
// device) sorted by decreasing key[list[i]] (asc = 0: key = qcnt, longest
// first) or increasing key[list[i]] (asc = 1: key = the C pairs' atom F);
// counting sort over kLptBuckets buckets, keys at or above the last bucket
// share it.
constexpr int kLptBuckets = 4096;
cudaError_t launch_lpt_order(const int* key, int asc, const int* list, int n_max, const long long* n_dev, int* hist,
                             int* out, cudaStream_t s);
int t1u_max_slots();
cudaError_t t1u_set_smem(int np);
// Needed V pairs: the second product's V store (MixPlan::Vm) and, with U.Vu
// set, the tcgen05 first product's V store, in one pass per pair.
cudaError_t launch_vstores(const DevPlan& P, const MixPlan& X, const T1UPlan& U, int np, const int* list, int n,
                           cudaStream_t s);
cudaError_t launch_t1u_stores(const DevPlan& P, const T1UPlan& U, int np, const int* qlist, int nq, bool dstore,
                              cudaStream_t s);
cudaError_t launch_t1_umma(const DevPlan& P, const MixPlan& X, const T1UPlan& U, int np, const int* qlist, int n,
                           size_t smem, int* work, int* err, cudaStream_t s);

// Split-precision kernels for n_ao up to 32 and n_abf up to 128 (hfx_wide.cu):
// warp-level MMAs on bf16 pieces copied from piece stores of D (plan), C (per
// call, from the FP64 blocks), Y (the Y build; offsets y_off, the split
// path's layout [alpha][z][rup16(n_ao(X))]) and Z (per pass); V and grad V FP64.
struct WideShapes {
  int MA = 0, MB = 0;          // n_abf rounded up to 16
  int KZ = 0;                  // n_ao rounded up to 16
  int t1_da = 0, t1_KC = 0;    // first product: a per range, columns (a, f) per range (rounded to 16)
  int t2_da = 0, t2_KC = 0;    // second product: a per range, columns (a, b) per range
  size_t smem_t1 = 0, smem_t2 = 0, smem_q2 = 0;
  bool ok = false;             // every shape fits the kernels' shared memory and tiles
};
long long wide_launch_count();
WideShapes wide_shapes(int np, int maxABF, int maxAO, size_t limit);
int wide_ybuild_row_blocks(int max_rows);
cudaError_t set_wide_smem_limits(int np);
// C pieces: per kept C pair, NP planes [alpha][rup8(n_ao(A) n_ao(F))] at Cw + cw_off[q]
long long wide_cpieces_size(int np, int n_abf, int n_ao_a, int n_ao_f);
cudaError_t launch_cpieces_w(const DevPlan& P, int np, uint16_t* Cw, const long long* cw_off, float* dCf,
                             cudaStream_t s);
cudaError_t launch_ybuild_w(const DevPlan& P, int np, uint16_t* Yp, const uint16_t* Cw, const long long* cw_off,
                            const uint16_t* Dw, const long long* dw_off, const int* ylist, const int* gX,
                            const int* gS, const int* gN, int ngroups, int RB, cudaStream_t s);
cudaError_t launch_term1_w(const DevPlan& P, int np, const uint16_t* Yp, const uint16_t* Cw, const long long* cw_off,
                           const uint16_t* Dw, const long long* dw_off, const float* dCf, const int* list, int n,
                           const WideShapes& w, cudaStream_t s);
// elements per bf16 piece plane of one pair slot of the Z store (rows (alpha, a), row stride KZ)
long long wide_zplane(int max_rows, int KZ);
// bf16 pieces of every D block (fixed for the plan): NP planes of
// rup16(n_ao(I)) x rup16(n_ao(J)) at Dw + dw_off[k] (multiples of 256)
cudaError_t launch_dsplit_w(const DevPlan& P, int np, uint16_t* Dw, const long long* dw_off, cudaStream_t s);
// Second product of the home atoms [a0, a1): k_term2_w over the pass's pair
// list (E, g^V and the Z piece store), then k_q2_w (grad C); slot0 as launch_term2_mma.
cudaError_t launch_term2_w(const DevPlan& P, int np, const uint16_t* Yp, uint16_t* Zw, const uint16_t* Dw,
                           const long long* dw_off, const float* dCf, const int* list, const long long* slot0, int n,
                           int a0, int a1, int max_rows, int max_c, const WideShapes& w, cudaStream_t s);

// Exclusive scan helpers.  `mode` selects what is summed per element i:
//   0: flag[i] != 0 (int32 flags)
//   1: flag[i] != 0 ? size[i] : 0
//   2: popcount-free "mask nonzero" over kMaskWords words (v_mask)
//   3: bytes[i] != 0
//   4: flag[i] itself (a count)
// The scan writes out[i] (exclusive prefix, int64) and *total (device).
// Device allocation hooks of a plan (hfx_options alloc / free; null = the
// CUDA runtime).
struct AllocHooks {
  void* (*alloc)(size_t, void*, void*) = nullptr;
  void (*free)(void*, size_t, void*, void*) = nullptr;
  void* ctx = nullptr;
  void* stream = nullptr;
  cudaError_t get(void** p, size_t bytes) const {
    if (!alloc) return cudaMalloc(p, bytes);
    *p = alloc(bytes, stream, ctx);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
  }
  void put(void* p, size_t bytes) const {
    if (!p) return;
    if (free) free(p, bytes, stream, ctx);
    else cudaFree(p);
  }
};

// Scratch of the scans.  A fixed ScanTmp (the no-allocation entry point's
// slice of the library's static array) is never freed or grown: a scan that
// needs more fails with cudaErrorMemoryAllocation.
struct ScanTmp {
  long long* buf = nullptr;
  size_t cap = 0;
  AllocHooks mem;
  bool fixed = false;
};
// long longs of scratch one scan_flags call over n elements needs
size_t scan_tmp_need(int n);
cudaError_t scan_flags(const int* flag, const long long* size, const unsigned* mask,
                       const unsigned char* bytes, int mode, int n, long long* out,
                       long long* total, ScanTmp& tmp, cudaStream_t s);
// list[out[i]] = base + i for every i selected by the same `mode` rule (a
// scan over a slice of a pair list passes the slice's first pair as base).
cudaError_t scatter_list(const int* flag, const unsigned* mask, const unsigned char* bytes, int mode,
                         int n, const long long* off, int* list, int base, cudaStream_t s);

}  // namespace hfx
