// Host side of libhfx: the C ABI, input validation, the periodic pair lists
// (atom I plus lattice vector R as one label, paper Eqs. 1-2), the dense
// lookup tables for D and Y blocks, device memory, and the order of the
// stages of one evaluation.  Every stage of the arithmetic runs in the CUDA
// kernels of hfx_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <limits>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "hfx.h"
#include "hfx_internal.h"

using hfx::DevPlan;
constexpr int kTot = 16;

namespace {

struct Failure {
  hfx_status status;
  std::string msg;
};

[[noreturn]] void fail(hfx_status s, const std::string& m) { throw Failure{s, m}; }

void ck(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  if (e == cudaErrorMemoryAllocation) fail(HFX_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
  fail(HFX_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Device allocation tracked by the plan (through the caller's hooks when
// hfx_options sets them).
struct DevMem {
  std::vector<std::pair<void*, size_t>> ptrs;
  long long bytes = 0;
  hfx::AllocHooks hooks;
  template <class T>
  T* alloc(size_t n) {
    if (n == 0) n = 1;
    void* p = nullptr;
    ck(hooks.get(&p, n * sizeof(T)), "device allocation");
    ptrs.emplace_back(p, n * sizeof(T));
    bytes += (long long)(n * sizeof(T));
    return static_cast<T*>(p);
  }
  void release(void* p) {
    for (auto it = ptrs.begin(); it != ptrs.end(); ++it)
      if (it->first == p) {
        hooks.put(p, it->second);
        bytes -= (long long)it->second;
        ptrs.erase(it);
        return;
      }
  }
  void free_all() {
    for (auto& q : ptrs) hooks.put(q.first, q.second);
    ptrs.clear();
    bytes = 0;
  }
};

template <class T>
void upload(T* dst, const std::vector<T>& src, cudaStream_t s) {
  if (!src.empty()) ck(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s), "H2D");
}

double det3(const double* L) {
  return L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) + L[2] * (L[3] * L[7] - L[4] * L[6]);
}

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Model radial function of V and its derivative (host copy for the radius).
void h_host(double r, double om, double& h, double& hp) {
  const double ec = std::erfc(om * r);
  h = ec / (r + 1.0);
  hp = (-2.0 * om / std::sqrt(M_PI)) * std::exp(-(om * r) * (om * r)) / (r + 1.0) - ec / ((r + 1.0) * (r + 1.0));
}

}  // namespace

struct hfx_plan {
  int dev = 0;
  cudaStream_t stream = nullptr;
  hfx_options opt{};
  int N = 0, S = 0;
  std::vector<int> species, n_ao, n_abf;
  double RC = 0, omega = 0, mmax = 0;
  bool aniso = false;
  double e[3] = {0, 0, 0};
  std::string err;
  DevMem mem;

  // host copies of D (for the lookup table and the D reach)
  std::vector<int> d_index;
  long long n_d = 0;

  // device model
  int *d_species = nullptr, *d_n_ao = nullptr, *d_n_abf = nullptr;
  long long *d_G_off = nullptr, *d_M_off = nullptr;
  double *d_G = nullptr, *d_Gp = nullptr, *d_M = nullptr, *d_Mnorm = nullptr, *d_Gmom = nullptr;
  float *d_Gf = nullptr, *d_Gpf = nullptr, *d_Mf = nullptr;
  double* d_Dval = nullptr;
  long long* d_Doff = nullptr;
  int* d_Didx = nullptr;
  double* d_Dkept = nullptr;
  bool dnorm_done = false;     // D norms taken (once per plan)
  long long d_kept = 0;
  int* d_dlut = nullptr;
  int HD[3] = {0, 0, 0};

  // lists (host side, at the reference geometry)
  std::vector<double> pos_ref, lat_ref;
  double list_Rabs = 0;    // largest |R_k| sum over listed pairs, for the staleness bound
  int nC = 0, nV = 0, nY = 0;
  int maxC = 0;
  int HY[3] = {0, 0, 0};
  bool lists_ready = false;
  bool frozen_ready = false;

  // device lists and per-call buffers
  std::vector<void*> list_bufs;   // freed on rebuild
  int *c_ptr = nullptr, *c_home = nullptr, *c_j = nullptr, *c_R = nullptr;
  long long* c_off = nullptr;
  double *Cst = nullptr, *dCst = nullptr, *c_norm = nullptr, *c_sc = nullptr;
  unsigned char* c_keep = nullptr;
  int *v_ptr = nullptr, *v_home = nullptr, *v_j = nullptr, *v_R = nullptr, *v_didx = nullptr;
  double* v_norm = nullptr;
  double* v_hg = nullptr;
  unsigned char *v_keep = nullptr, *v_t2 = nullptr;
  unsigned* v_mask = nullptr;
  int* v_flag = nullptr;
  long long *v_off = nullptr, *v_size = nullptr, *v_idx = nullptr, *t1_idx = nullptr, *t2_idx = nullptr;
  int *v_list = nullptr, *t1_list = nullptr, *t2_list = nullptr;
  int *y_ptr = nullptr, *y_home = nullptr, *y_j = nullptr, *y_R = nullptr, *ylut = nullptr;
  double* yhat = nullptr;
  int* y_flag = nullptr;
  long long *y_off = nullptr, *y_size = nullptr, *y_idx = nullptr;
  int* y_list = nullptr;
  double *gC = nullptr, *gV = nullptr;
  unsigned long long* fx = nullptr;   // deterministic plans: exact cells of gC, gV, E and the virial, F
  size_t fx_words = 0;
  long long c_elems = 0;

  // per-call state
  double* d_pos = nullptr;
  double* d_lat = nullptr;     // [9] lattice of the current call
  double* d_out = nullptr;     // [1 + 3N + 9]
  double* d_acc = nullptr;     // hfx::ACC_N
  long long* d_tot = nullptr;  // [kTot] totals of the scans, then hfx::CNT_N counters
  int* d_err = nullptr;        // set by a kernel whose bounded wait ran out
  std::vector<std::pair<int, int>> chunks;   // passes of home atoms [a0, a1)
  std::vector<long long> ctot;               // per-pass totals of the last screening (kCT each)
  std::vector<int> c_ptr_h, v_ptr_h;         // host copies of the list offsets per atom
  bool has_ref = false;                      // reference result of hfx_set_reference
  std::vector<double> ref;                   // [E, F (3N), sigma (9)]
  double* Yst = nullptr;
  long long Ycap = 0;
  double* Vst = nullptr;
  long long Vcap = 0;
  hfx::ScanTmp scan_tmp;
  long long tot[16] = {0};     // y elems, y count, v elems, v count, t1, t2, triplets, t1q, vm elems
  unsigned long long cnt[hfx::CNT_N] = {0};

  // kernel shapes
  int beta_chunk = 1, alpha_chunk = 1;
  size_t smem_t1 = 0, smem_t2 = 0;

  // split-precision path (np = bf16 pieces per operand; 0 = FP64 path)
  int np = 0;
  uint16_t* Dsp = nullptr;
  long long* dsp_off = nullptr;
  uint16_t* Ysp = nullptr;
  long long Yspcap = 0;
  uint16_t* Cm = nullptr;
  long long* cm_off = nullptr;
  int *gcnt = nullptr, *gX = nullptr, *gS = nullptr, *gN = nullptr;   // groups of needed Y keys
  long long* goff = nullptr;
  uint16_t* Vm = nullptr;
  long long Vmcap = 0;
  long long *vm_off = nullptr, *vm_size = nullptr;
  int* qcnt = nullptr;
  long long *qoff = nullptr, *q_idx = nullptr;
  int* t1q_list = nullptr;
  int* t1q_lpt = nullptr;      // the same items, longest (most kept B) first
  int t1_order = 0;            // first-product items: 0 longest first, 1 home-atom (list) order, 2 by F
  int ybtpc = 2, q2tpc = 2;    // 128-row tiles per CTA of the tcgen05 Y build and Q2 GEMM (autotuner);
                               // q2tpc = 3: two tiles, one CTA per SM with the deep pipeline
  int q2_flush = 32;           // pairs per FP32 run of the second product's Q2 accumulator (128 for BF16X6)
  uint16_t* YspT = nullptr;    // transposed Y pieces (second product)
  long long YspTcap = 0;
  int* ytab = nullptr;         // D-block tables of the Y build and the second product
  int* q2tab = nullptr;
  long long ytabcap = 0, q2tabcap = 0;
  int* lpt_hist = nullptr;
  int* blist = nullptr;
  long long blist_cap = 0;
  int MAmax = 0, MBmax = 0, KSmax = 0, YRmax = 0, ZROWS = 0, KZmax = 0, FC = 0, MC = 0;
  long long zblk = 0;
  uint16_t* Zst = nullptr;
  long long Zcap = 0;
  hfx::DRows drows{};          // tensor map of the D piece rows
  int maxV = 0;                  // most V-pair candidates of one home atom
  size_t smem_m1 = 0, smem_m2 = 0;
  // tcgen05 first product (n_abf <= 64, n_ao <= 16): operand stores and shape
  bool t1u = false;
  int t1u_KP = 0, t1u_NS = 0, t1u_FS = 1, t1u_seg = 32;
  size_t t1u_limit = 0;        // dynamic shared memory the Y ring may fill up to
  size_t smem_t1u = 0;
  uint16_t* Cu = nullptr;
  long long Cucap = 0;
  uint16_t* Vu = nullptr;
  long long Vucap = 0;
  float* Yf = nullptr;
  long long Yfcap = 0;
  float* Df = nullptr;
  int* d_work = nullptr;       // item counter of the tcgen05 first-product kernel
  // tcgen05 R2 / Z of the second product (same shapes): core-matrix Y stores, V store per pair slot
  bool t2u = false;
  size_t smem_t2u = 0;
  uint16_t* Vz = nullptr;
  long long Vzcap = 0;
  // split path for n_ao > 16 (hfx_wide.cu): FP64 C, V and D blocks, FP32 Y store
  bool wide = false;
  hfx::WideShapes ws{};
  int wide_RB = 0;             // 64-row blocks of the largest Y block
  int wide_maxrows = 0;        // most rows (alpha, a) of a C block
  uint16_t* Cw = nullptr;      // C pieces of every C pair (written per call)
  float* dCf = nullptr;        // grad C of every C pair in FP32, the layout of dCst (written per call)
  long long* cw_off = nullptr;
  uint16_t* Zw = nullptr;      // Z^{AB} of one pass's second-product pairs (bf16 pieces)
  long long Zwcap = 0;
  uint16_t* Dw = nullptr;      // bf16 pieces of every D block (fixed for the plan)
  long long* dw_off = nullptr;

  bool timing = false;
  bool noalloc_call = false;   // set only inside hfx_energy_force_stress_noalloc
  cudaGraphExec_t gexec = nullptr;   // recorded evaluation of a frozen plan (hfx_options.graph)
  cudaStream_t cap_stream = nullptr; // the stream it is recorded on (the legacy stream cannot be captured)
  long long graph_launches = 0;      // kernels in it
  std::vector<double> pos_host_buf;
  hfx_stats last{};

  template <class T>
  T* lalloc(size_t n) {
    T* p = mem.alloc<T>(n);
    list_bufs.push_back(p);
    return p;
  }
  void free_lists() {
    for (void* p : list_bufs) mem.release(p);
    list_bufs.clear();
  }
};

namespace {

void validate_options(const hfx_options* o) {
  if (!o) fail(HFX_ERR_INVALID, "options is NULL");
  const double th[6] = {o->theta_C, o->theta_dC, o->theta_V, o->theta_dV, o->theta_D, o->theta_CS};
  for (double t : th)
    if (!std::isfinite(t) || t < 0) fail(HFX_ERR_INVALID, "thresholds must be finite and >= 0");
  if (o->precision != HFX_FP64 && o->precision != HFX_BF16X3 && o->precision != HFX_BF16X6)
    fail(HFX_ERR_UNSUPPORTED, "precision must be HFX_FP64, HFX_BF16X3 or HFX_BF16X6");
  if (o->terms < 1 || o->terms > 3) fail(HFX_ERR_INVALID, "terms must be 1, 2 or 3");
  if (!std::isfinite(o->skin) || o->skin < 0) fail(HFX_ERR_INVALID, "skin must be finite and >= 0");
  if (o->home_chunk < 0) fail(HFX_ERR_INVALID, "home_chunk must be >= 0");
  if (o->graph != 0 && o->graph != 1) fail(HFX_ERR_INVALID, "graph must be 0 or 1");
  if ((o->alloc == nullptr) != (o->free == nullptr)) fail(HFX_ERR_INVALID, "alloc and free must be set together");
}

void validate_geometry(int N, const double* lattice, const double* positions) {
  if (!lattice || !positions) fail(HFX_ERR_INVALID, "lattice or positions is NULL");
  if (!finite_all(lattice, 9) || !finite_all(positions, (size_t)N * 3))
    fail(HFX_ERR_INVALID, "non-finite lattice or positions");
  if (std::fabs(det3(lattice)) < 1e-9) fail(HFX_ERR_INVALID, "singular lattice");
}

void upload_model(hfx_plan* P, const hfx_system* sys, const hfx_model* m) {
  const int S = m->n_species, N = sys->n_atoms;
  cudaStream_t s = P->stream;
  P->species.assign(sys->species, sys->species + N);
  P->n_ao.assign(m->n_ao, m->n_ao + S);
  P->n_abf.assign(m->n_abf, m->n_abf + S);
  for (int i = 0; i < N; ++i)
    if (P->species[i] < 0 || P->species[i] >= S) fail(HFX_ERR_INVALID, "species out of range");
  for (int t = 0; t < S; ++t) {
    if (P->n_ao[t] < 1 || P->n_ao[t] > hfx::kMaxAO) fail(HFX_ERR_INVALID, "n_ao out of range 1..32");
    if (P->n_abf[t] < 1 || P->n_abf[t] > hfx::kMaxABF) fail(HFX_ERR_INVALID, "n_abf out of range 1..128");
  }
  std::vector<long long> goff(S * S), moff(S * S);
  long long gsz = 0, msz = 0;
  for (int a = 0; a < S; ++a)
    for (int b = 0; b < S; ++b) {
      goff[a * S + b] = gsz;
      moff[a * S + b] = msz;
      gsz += (long long)P->n_abf[a] * P->n_ao[a] * P->n_ao[b];
      msz += (long long)P->n_abf[a] * P->n_abf[b];
    }
  std::vector<double> G(gsz), M(msz), Gp, Mnorm(S * S), Gmom(3 * S * S, 0.0);
  if (m->G_aniso) Gp.resize(gsz);
  double mmax = 0;
  for (int a = 0; a < S; ++a)
    for (int b = 0; b < S; ++b) {
      const long long ng = (long long)P->n_abf[a] * P->n_ao[a] * P->n_ao[b];
      const long long nm = (long long)P->n_abf[a] * P->n_abf[b];
      if (!m->G[a * S + b] || !m->M[a * S + b]) fail(HFX_ERR_INVALID, "NULL template");
      std::memcpy(&G[goff[a * S + b]], m->G[a * S + b], ng * sizeof(double));
      std::memcpy(&M[moff[a * S + b]], m->M[a * S + b], nm * sizeof(double));
      if (m->G_aniso) {
        if (!m->G_aniso[a * S + b]) fail(HFX_ERR_INVALID, "NULL anisotropic template");
        std::memcpy(&Gp[goff[a * S + b]], m->G_aniso[a * S + b], ng * sizeof(double));
      }
      double s2 = 0;
      for (long long k = 0; k < nm; ++k) s2 += M[moff[a * S + b] + k] * M[moff[a * S + b] + k];
      double* gm = &Gmom[3 * (a * S + b)];   // moments of the C templates (closed-form C norms)
      for (long long k = 0; k < ng; ++k) {
        const double gv = G[goff[a * S + b] + k], gq = m->G_aniso ? Gp[goff[a * S + b] + k] : 0.0;
        gm[0] += gv * gv;
        gm[1] += gv * gq;
        gm[2] += gq * gq;
      }
      Mnorm[a * S + b] = std::sqrt(s2);
      mmax = std::max(mmax, Mnorm[a * S + b]);
    }
  if (!finite_all(G.data(), G.size()) || !finite_all(M.data(), M.size()) || !finite_all(Gp.data(), Gp.size()))
    fail(HFX_ERR_INVALID, "non-finite template");
  // V_BA = V_AB^T needs M_ts = M_st^T (Sec. 3.1)
  for (int a = 0; a < S; ++a)
    for (int b = 0; b < S; ++b)
      for (int x = 0; x < P->n_abf[a]; ++x)
        for (int y = 0; y < P->n_abf[b]; ++y) {
          const double u = M[moff[a * S + b] + (long long)x * P->n_abf[b] + y];
          const double v = M[moff[b * S + a] + (long long)y * P->n_abf[a] + x];
          if (std::fabs(u - v) > 1e-12 * (1.0 + std::fabs(u))) fail(HFX_ERR_INVALID, "M_ts != M_st^T");
        }
  P->mmax = mmax;
  P->d_species = P->mem.alloc<int>(N);
  P->d_n_ao = P->mem.alloc<int>(S);
  P->d_n_abf = P->mem.alloc<int>(S);
  P->d_G_off = P->mem.alloc<long long>(S * S);
  P->d_M_off = P->mem.alloc<long long>(S * S);
  P->d_G = P->mem.alloc<double>(gsz);
  P->d_M = P->mem.alloc<double>(msz);
  P->d_Mnorm = P->mem.alloc<double>(S * S);
  P->d_Gmom = P->mem.alloc<double>(3 * S * S);
  upload(P->d_species, P->species, s);
  upload(P->d_n_ao, P->n_ao, s);
  upload(P->d_n_abf, P->n_abf, s);
  upload(P->d_G_off, goff, s);
  upload(P->d_M_off, moff, s);
  upload(P->d_G, G, s);
  upload(P->d_M, M, s);
  upload(P->d_Mnorm, Mnorm, s);
  upload(P->d_Gmom, Gmom, s);
  // kept alive until the stream synchronisation below
  const std::vector<float> Gf(G.begin(), G.end()), Mf(M.begin(), M.end()), Gpf(Gp.begin(), Gp.end());
  P->d_Gf = P->mem.alloc<float>(gsz);
  P->d_Mf = P->mem.alloc<float>(msz);
  upload(P->d_Gf, Gf, s);
  upload(P->d_Mf, Mf, s);
  if (m->G_aniso) {
    P->d_Gp = P->mem.alloc<double>(gsz);
    upload(P->d_Gp, Gp, s);
    P->d_Gpf = P->mem.alloc<float>(gsz);
    upload(P->d_Gpf, Gpf, s);
    P->aniso = true;
    for (int k = 0; k < 3; ++k) P->e[k] = m->aniso_dir[k];
    if (!finite_all(P->e, 3)) fail(HFX_ERR_INVALID, "non-finite anisotropy direction");
  }
  ck(cudaStreamSynchronize(s), "upload model");
}

// D blocks: validation, the dense (i, j, R) lookup table, device copies.
void upload_density(hfx_plan* P, const hfx_model* m) {
  const int N = P->N;
  const long long nd = m->n_d;
  if (nd < 0) fail(HFX_ERR_INVALID, "n_d < 0");
  if (nd > 0 && (!m->d_index || !m->d_offset || !m->d_values)) fail(HFX_ERR_INVALID, "NULL D arrays");
  P->n_d = nd;
  P->d_index.assign(m->d_index, m->d_index + 5 * nd);
  std::vector<long long> off(m->d_offset, m->d_offset + nd + 1);
  if (off[0] != 0) fail(HFX_ERR_INVALID, "d_offset[0] != 0");
  int H[3] = {0, 0, 0};
  for (long long k = 0; k < nd; ++k) {
    const int* r = &P->d_index[5 * k];
    if (r[0] < 0 || r[0] >= N || r[1] < 0 || r[1] >= N) fail(HFX_ERR_INVALID, "D atom index out of range");
    const long long want = (long long)P->n_ao[P->species[r[0]]] * P->n_ao[P->species[r[1]]];
    if (off[k + 1] - off[k] != want) fail(HFX_ERR_INVALID, "D block size != n_ao(I)*n_ao(J)");
    for (int c = 0; c < 3; ++c) {
      if (std::abs(r[2 + c]) > 1000) fail(HFX_ERR_INVALID, "D image index too large");
      H[c] = std::max(H[c], std::abs(r[2 + c]));
    }
  }
  const long long nvals = off[nd];
  if (!finite_all(m->d_values, (size_t)nvals)) fail(HFX_ERR_INVALID, "non-finite D values");
  for (int c = 0; c < 3; ++c) P->HD[c] = H[c];
  const long long n0 = 2 * H[0] + 1, n1 = 2 * H[1] + 1, n2 = 2 * H[2] + 1;
  const long long lut_n = (long long)N * N * n0 * n1 * n2;
  if (lut_n > (1ll << 31)) fail(HFX_ERR_UNSUPPORTED, "D lookup table too large");
  std::vector<int> lut(lut_n, -1);
  auto lidx = [&](int i, int j, int a, int b, int c) {
    return ((((long long)i * N + j) * n0 + (a + H[0])) * n1 + (b + H[1])) * n2 + (c + H[2]);
  };
  for (long long k = 0; k < nd; ++k) {
    const int* r = &P->d_index[5 * k];
    int& slot = lut[lidx(r[0], r[1], r[2], r[3], r[4])];
    if (slot != -1) fail(HFX_ERR_INVALID, "duplicate D block");
    slot = (int)k;
  }
  // both orientations, D_JI(-R) = D_IJ(R)^T (needed by the symmetric exchange products)
  for (long long k = 0; k < nd; ++k) {
    const int* r = &P->d_index[5 * k];
    const int t = lut[lidx(r[1], r[0], -r[2], -r[3], -r[4])];
    if (t < 0) fail(HFX_ERR_INVALID, "D_JI(-R) missing for a given D_IJ(R)");
    const int na = P->n_ao[P->species[r[0]]], nb = P->n_ao[P->species[r[1]]];
    for (int x = 0; x < na; ++x)
      for (int y = 0; y < nb; ++y) {
        const double u = m->d_values[off[k] + (long long)x * nb + y];
        const double v = m->d_values[off[t] + (long long)y * na + x];
        if (std::fabs(u - v) > 1e-12 * (1.0 + std::fabs(u))) fail(HFX_ERR_INVALID, "D_JI(-R) != D_IJ(R)^T");
      }
  }
  cudaStream_t s = P->stream;
  P->d_Dval = P->mem.alloc<double>(nvals);
  P->d_Doff = P->mem.alloc<long long>(nd + 1);
  P->d_Didx = P->mem.alloc<int>(5 * nd);
  P->d_Dkept = P->mem.alloc<double>(nd);
  P->d_dlut = P->mem.alloc<int>(lut_n);
  if (nvals) ck(cudaMemcpyAsync(P->d_Dval, m->d_values, nvals * sizeof(double), cudaMemcpyHostToDevice, s), "H2D D");
  upload(P->d_Doff, off, s);
  upload(P->d_Didx, P->d_index, s);
  upload(P->d_dlut, lut, s);
  ck(cudaStreamSynchronize(s), "upload D");
}

double v_radius(const hfx_plan* P) {
  const double tv = P->opt.theta_V, tdv = P->opt.theta_dV;
  if (tv <= 0 && tdv <= 0) return std::numeric_limits<double>::infinity();
  auto above = [&](double r) {
    double h, hp;
    h_host(r, P->omega, h, hp);
    return P->mmax * h > tv || P->mmax * std::fabs(hp) > tdv;
  };
  double lo = 0, hi = 1;
  while (above(hi) && hi < 1e6) hi *= 2;
  for (int it = 0; it < 80; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (above(mid)) lo = mid;
    else hi = mid;
  }
  return hi + 1.0;
}

DevPlan make_devplan(hfx_plan* P, const double* lattice) {
  DevPlan D{};
  D.N = P->N;
  D.S = P->S;
  D.species = P->d_species;
  D.n_ao = P->d_n_ao;
  D.n_abf = P->d_n_abf;
  D.G_off = P->d_G_off;
  D.G = P->d_G;
  D.Gp = P->aniso ? P->d_Gp : nullptr;
  D.M_off = P->d_M_off;
  D.M = P->d_M;
  D.Gf = P->d_Gf;
  D.Gpf = P->aniso ? P->d_Gpf : nullptr;
  D.Mf = P->d_Mf;
  D.Mnorm = P->d_Mnorm;
  D.Gmom = P->d_Gmom;
  for (int k = 0; k < 3; ++k) D.e[k] = P->e[k];
  D.RC = P->RC;
  D.omega = P->omega;
  D.thC = P->opt.theta_C;
  D.thdC = P->opt.theta_dC;
  D.thV = P->opt.theta_V;
  D.thdV = P->opt.theta_dV;
  D.thD = P->opt.theta_D;
  D.thCS = P->opt.theta_CS;
  D.terms = P->opt.terms;
  D.h0 = P->chunks.empty() ? 0 : P->chunks.front().first;
  D.h1 = P->chunks.empty() ? P->N : P->chunks.back().second;
  D.pos = P->d_pos;
  D.L = P->d_lat;   // the entry points copy the call's lattice there first
  D.n_d = P->n_d;
  D.Dval = P->d_Dval;
  D.Doff = P->d_Doff;
  D.Didx = P->d_Didx;
  D.Dkept = P->d_Dkept;
  D.dlut = P->d_dlut;
  D.HD0 = P->HD[0];
  D.HD1 = P->HD[1];
  D.HD2 = P->HD[2];
  D.nC = P->nC;
  D.c_ptr = P->c_ptr;
  D.c_home = P->c_home;
  D.c_j = P->c_j;
  D.c_R = P->c_R;
  D.c_off = P->c_off;
  D.Cst = P->Cst;
  D.c_sc = P->c_sc;
  D.dCst = P->dCst;
  D.c_norm = P->c_norm;
  D.c_keep = P->c_keep;
  D.nV = P->nV;
  D.v_ptr = P->v_ptr;
  D.v_home = P->v_home;
  D.v_j = P->v_j;
  D.v_R = P->v_R;
  D.v_didx = P->v_didx;
  D.v_norm = P->v_norm;
  D.v_hg = P->v_hg;
  D.v_keep = P->v_keep;
  D.v_mask = P->v_mask;
  D.v_t2 = P->v_t2;
  D.v_flag = P->v_flag;
  D.v_off = P->v_off;
  D.Vst = P->Vst;
  D.nY = P->nY;
  D.y_ptr = P->y_ptr;
  D.y_home = P->y_home;
  D.y_j = P->y_j;
  D.y_R = P->y_R;
  D.yhat = P->yhat;
  D.y_flag = P->y_flag;
  D.y_off = P->y_off;
  D.Yst = P->Yst;
  D.ylut = P->ylut;
  D.HY0 = P->HY[0];
  D.HY1 = P->HY[1];
  D.HY2 = P->HY[2];
  D.gC = P->gC;
  D.gV = P->gV;
  D.acc = P->d_acc;
  if (P->fx) {   // [gC 3 nC][gV 3 nV][E, virial 10][F 3N] cells of two words
    D.fxC = P->fx;
    D.fxV = D.fxC + 2 * 3 * (size_t)P->nC;
    D.fxA = D.fxV + 2 * 3 * (size_t)P->nV;
    D.fxF = D.fxA + 2 * 10;
  }
  D.cnt = reinterpret_cast<unsigned long long*>(P->d_tot + kTot);
  return D;
}

// Pair lists (K0): C pairs within R_C + skin, V pairs within the V radius
// (capped at R_C + D reach + 1) + skin, Y keys within R_C + D reach + skin.
void build_lists(hfx_plan* P, const double* L, const double* pos) {
  const int N = P->N;
  // D reach at this geometry
  double rd = 0;
  for (long long k = 0; k < P->n_d; ++k) {
    const int* r = &P->d_index[5 * k];
    double d2 = 0;
    for (int c = 0; c < 3; ++c) {
      const double dv = pos[3 * r[1] + c] + r[2] * L[c] + r[3] * L[3 + c] + r[4] * L[6 + c] - pos[3 * r[0] + c];
      d2 += dv * dv;
    }
    rd = std::max(rd, std::sqrt(d2));
  }
  const double skin = P->opt.skin;
  const double rC = P->RC + skin;
  const double rV = std::min(v_radius(P), P->RC + rd + 1.0) + skin;
  const double rY = P->RC + rd + skin;
  const double rmax = std::max(rC, std::max(rV, rY));
  // reciprocal vectors: rows of inv(L)^T
  const double det = det3(L);
  double B[9];
  B[0] = (L[4] * L[8] - L[5] * L[7]) / det;
  B[1] = (L[5] * L[6] - L[3] * L[8]) / det;
  B[2] = (L[3] * L[7] - L[4] * L[6]) / det;
  B[3] = (L[2] * L[7] - L[1] * L[8]) / det;
  B[4] = (L[0] * L[8] - L[2] * L[6]) / det;
  B[5] = (L[1] * L[6] - L[0] * L[7]) / det;
  B[6] = (L[1] * L[5] - L[2] * L[4]) / det;
  B[7] = (L[2] * L[3] - L[0] * L[5]) / det;
  B[8] = (L[0] * L[4] - L[1] * L[3]) / det;
  // Candidates by a cell list over the wrapped fractional coordinates:
  // atom i sits at w_i = pos_i - L k_i with k_i = floor(s_i), s_i = B pos_i;
  // cells are at least max(rmax / 8, 1 A) wide (n_k per axis, the D reach
  // makes rmax ~30 A on the Si cells); atom A searches the cells within
  // +-m_k of its own, where m_k = ceil(n_k rmax |b_k|) covers
  // every fractional separation |ds_k| <= rmax |b_k| of two points within
  // rmax.  A visited cell c (unwrapped) is cell c mod n of image floor(c / n)
  // in wrapped coordinates, i.e. image R = floor(c / n) - k_j + k_A of the
  // original positions; each (j, R) is visited at most once.  The inclusion
  // test below is the direct one on the original positions, and each atom's
  // candidates are sorted by (j, R), so the lists do not depend on the
  // binning.
  int ncell[3], mc[3];
  double bnorm[3];
  for (int k = 0; k < 3; ++k) {
    bnorm[k] = std::sqrt(B[3 * k] * B[3 * k] + B[3 * k + 1] * B[3 * k + 1] + B[3 * k + 2] * B[3 * k + 2]);
    const double width = 1.0 / bnorm[k];   // distance between the lattice planes of axis k
    ncell[k] = std::max(1, std::min(256, (int)std::floor(width / std::max(0.125 * rmax, 1.0))));
    mc[k] = (int)std::ceil(ncell[k] * rmax * bnorm[k]);
    if (mc[k] > 200 * ncell[k]) fail(HFX_ERR_UNSUPPORTED, "pair range spans too many images");
  }
  std::vector<int> kimg(3 * (size_t)N), cell_of(N);
  const int nct = ncell[0] * ncell[1] * ncell[2];
  std::vector<int> cell_ptr(nct + 1, 0), cell_atoms(N);
  std::vector<double> wpos(3 * (size_t)N);
  for (int i = 0; i < N; ++i) {
    int ci[3];
    for (int k = 0; k < 3; ++k) {
      const double sk = B[3 * k] * pos[3 * i] + B[3 * k + 1] * pos[3 * i + 1] + B[3 * k + 2] * pos[3 * i + 2];
      const double fk = std::floor(sk);
      kimg[3 * i + k] = (int)fk;
      ci[k] = std::min(ncell[k] - 1, std::max(0, (int)std::floor((sk - fk) * ncell[k])));
    }
    for (int k = 0; k < 3; ++k)
      wpos[3 * i + k] = pos[3 * i + k] - (kimg[3 * i] * L[k] + kimg[3 * i + 1] * L[3 + k] + kimg[3 * i + 2] * L[6 + k]);
    cell_of[i] = (ci[0] * ncell[1] + ci[1]) * ncell[2] + ci[2];
    ++cell_ptr[cell_of[i] + 1];
  }
  for (int c = 0; c < nct; ++c) cell_ptr[c + 1] += cell_ptr[c];
  {
    std::vector<int> fill(cell_ptr.begin(), cell_ptr.end() - 1);
    for (int i = 0; i < N; ++i) cell_atoms[fill[cell_of[i]]++] = i;
  }
  auto floordiv = [](int a, int n) { return a >= 0 ? a / n : -((-a + n - 1) / n); };
  struct Cand {
    int j, a, b, c;
  };
  std::vector<Cand> cand;
  std::vector<int> c_ptr(N + 1, 0), v_ptr(N + 1, 0), y_ptr(N + 1, 0);
  std::vector<int> c_home, c_j, c_R, v_home, v_j, v_R, y_home, y_j, y_R;
  int HY[3] = {0, 0, 0};
  double Rabs = 0;
  const double rmax2 = (rmax * 1.0001 + 1e-9) * (rmax * 1.0001 + 1e-9);
  for (int A = 0; A < N; ++A) {
    c_ptr[A] = (int)c_j.size();
    v_ptr[A] = (int)v_j.size();
    y_ptr[A] = (int)y_j.size();
    const int cA = cell_of[A];
    const int cA0 = cA / (ncell[1] * ncell[2]), cA1 = (cA / ncell[2]) % ncell[1], cA2 = cA % ncell[2];
    cand.clear();
    for (int d0 = -mc[0]; d0 <= mc[0]; ++d0)
      for (int d1 = -mc[1]; d1 <= mc[1]; ++d1)
        for (int d2 = -mc[2]; d2 <= mc[2]; ++d2) {
          const int u0 = cA0 + d0, u1 = cA1 + d1, u2 = cA2 + d2;
          const int W0 = floordiv(u0, ncell[0]), W1 = floordiv(u1, ncell[1]), W2 = floordiv(u2, ncell[2]);
          const int cw = ((u0 - W0 * ncell[0]) * ncell[1] + (u1 - W1 * ncell[1])) * ncell[2] + (u2 - W2 * ncell[2]);
          for (int t = cell_ptr[cw]; t < cell_ptr[cw + 1]; ++t) {
            const int j = cell_atoms[t];
            double e2 = 0;   // loose prefilter in wrapped coordinates
            for (int k = 0; k < 3; ++k) {
              const double dv = wpos[3 * j + k] + W0 * L[k] + W1 * L[3 + k] + W2 * L[6 + k] - wpos[3 * A + k];
              e2 += dv * dv;
            }
            if (e2 > rmax2) continue;
            cand.push_back({j, W0 - kimg[3 * j] + kimg[3 * A], W1 - kimg[3 * j + 1] + kimg[3 * A + 1],
                            W2 - kimg[3 * j + 2] + kimg[3 * A + 2]});
          }
        }
    std::sort(cand.begin(), cand.end(), [](const Cand& x, const Cand& y) {
      if (x.j != y.j) return x.j < y.j;
      if (x.a != y.a) return x.a < y.a;
      if (x.b != y.b) return x.b < y.b;
      return x.c < y.c;
    });
    for (const Cand& q : cand) {
      const int j = q.j, a = q.a, b = q.b, c = q.c;
      {
            double d2 = 0;
            for (int k = 0; k < 3; ++k) {
              const double dv = (pos[3 * j + k] + (a * L[k] + b * L[3 + k] + c * L[6 + k])) - pos[3 * A + k];
              d2 += dv * dv;
            }
            const double r = std::sqrt(d2);
            const bool inC = r < rC, inV = r < rV, inY = r < rY;
            if (!(inC || inV || inY)) continue;
            Rabs = std::max(Rabs, (double)(std::abs(a) + std::abs(b) + std::abs(c)));
            if (inC) {
              c_home.push_back(A);
              c_j.push_back(j);
              c_R.insert(c_R.end(), {a, b, c});
            }
            if (inV) {
              v_home.push_back(A);
              v_j.push_back(j);
              v_R.insert(v_R.end(), {a, b, c});
            }
            if (inY) {
              y_home.push_back(A);
              y_j.push_back(j);
              y_R.insert(y_R.end(), {a, b, c});
              HY[0] = std::max(HY[0], std::abs(a));
              HY[1] = std::max(HY[1], std::abs(b));
              HY[2] = std::max(HY[2], std::abs(c));
            }
      }
    }
    if ((int)c_j.size() - c_ptr[A] > hfx::kMaxCPerAtom)
      fail(HFX_ERR_UNSUPPORTED, "more than 256 C-pair candidates on one atom");
  }
  c_ptr[N] = (int)c_j.size();
  v_ptr[N] = (int)v_j.size();
  y_ptr[N] = (int)y_j.size();
  const int nC = c_ptr[N], nV = v_ptr[N], nY = y_ptr[N];
  int maxC = 0, maxV = 0;
  for (int A = 0; A < N; ++A) {
    maxC = std::max(maxC, c_ptr[A + 1] - c_ptr[A]);
    maxV = std::max(maxV, v_ptr[A + 1] - v_ptr[A]);
  }
  // D block of each V pair, Y-key lookup table
  const long long n0 = 2 * P->HD[0] + 1, n1 = 2 * P->HD[1] + 1, n2 = 2 * P->HD[2] + 1;
  std::vector<int> v_didx(nV, -1);
  {
    std::vector<int> dl((size_t)N * N * n0 * n1 * n2);
    ck(cudaMemcpy(dl.data(), P->d_dlut, dl.size() * sizeof(int), cudaMemcpyDeviceToHost), "D2H dlut");
    for (int p = 0; p < nV; ++p) {
      const int a = v_R[3 * p], b = v_R[3 * p + 1], c = v_R[3 * p + 2];
      if (std::abs(a) > P->HD[0] || std::abs(b) > P->HD[1] || std::abs(c) > P->HD[2]) continue;
      v_didx[p] = dl[((((long long)v_home[p] * N + v_j[p]) * n0 + (a + P->HD[0])) * n1 + (b + P->HD[1])) * n2 +
                     (c + P->HD[2])];
    }
  }
  const long long m0 = 2 * HY[0] + 1, m1 = 2 * HY[1] + 1, m2 = 2 * HY[2] + 1;
  const long long ylut_n = (long long)N * N * m0 * m1 * m2;
  if (ylut_n > (1ll << 31)) fail(HFX_ERR_UNSUPPORTED, "Y lookup table too large");
  std::vector<int> ylut(ylut_n, -1);
  for (int y = 0; y < nY; ++y) {
    const long long idx = ((((long long)y_home[y] * N + y_j[y]) * m0 + (y_R[3 * y] + HY[0])) * m1 +
                           (y_R[3 * y + 1] + HY[1])) * m2 + (y_R[3 * y + 2] + HY[2]);
    ylut[idx] = y;
  }
  std::vector<long long> c_off(nC + 1, 0), v_size(nV), y_size(nY);
  for (int p = 0; p < nC; ++p) {
    const int sA = P->species[c_home[p]], sj = P->species[c_j[p]];
    c_off[p + 1] = c_off[p] + (long long)P->n_abf[sA] * P->n_ao[sA] * P->n_ao[sj];
  }
  for (int p = 0; p < nV; ++p)
    v_size[p] = 4ll * P->n_abf[P->species[v_home[p]]] * P->n_abf[P->species[v_j[p]]];
  for (int y = 0; y < nY; ++y) {
    const int sX = P->species[y_home[y]], sz = P->species[y_j[y]];
    if (P->t2u)  // bf16 pieces of 64 rows alpha x (z, x) columns in core-matrix order
      y_size[y] = (long long)P->np * 64 * 16 * P->n_ao[sz];
    else if (P->np)  // bf16 pieces of [alpha][z][rup16(n_ao(X))]
      y_size[y] = (long long)P->np * P->n_abf[sX] * P->n_ao[sz] * ((P->n_ao[sX] + 15) / 16 * 16);
    else
      y_size[y] = (long long)P->n_abf[sX] * P->n_ao[sX] * P->n_ao[sz];
  }

  // (re)allocate list buffers
  P->free_lists();
  P->nC = nC;
  P->nV = nV;
  P->nY = nY;
  P->maxC = maxC;
  P->maxV = maxV;
  for (int k = 0; k < 3; ++k) P->HY[k] = HY[k];
  P->c_elems = c_off[nC];
  cudaStream_t s = P->stream;
  P->c_ptr = P->lalloc<int>(N + 1);
  P->c_home = P->lalloc<int>(nC);
  P->c_j = P->lalloc<int>(nC);
  P->c_R = P->lalloc<int>(3 * (size_t)nC);
  P->c_off = P->lalloc<long long>(nC + 1);
  // FP64 C blocks: the FP64 path and the wide split path only (the other
  // split path evaluates C from the model where it writes its operand stores)
  const bool fp64_c = !P->np || P->wide;
  P->Cst = P->lalloc<double>(fp64_c ? P->c_elems : 1);
  P->c_sc = P->lalloc<double>(8 * (size_t)nC);
  P->dCst = P->lalloc<double>(fp64_c ? 3 * P->c_elems : 1);
  P->c_norm = P->lalloc<double>(nC);
  P->c_keep = P->lalloc<unsigned char>(nC);
  P->v_ptr = P->lalloc<int>(N + 1);
  P->v_home = P->lalloc<int>(nV);
  P->v_j = P->lalloc<int>(nV);
  P->v_R = P->lalloc<int>(3 * (size_t)nV);
  P->v_didx = P->lalloc<int>(nV);
  P->v_norm = P->lalloc<double>(nV);
  P->v_hg = P->lalloc<double>(4 * (size_t)nV);
  P->v_keep = P->lalloc<unsigned char>(nV);
  P->v_t2 = P->lalloc<unsigned char>(nV);
  P->v_mask = P->lalloc<unsigned>((size_t)nV * hfx::kMaskWords);
  P->v_flag = P->lalloc<int>(nV);
  P->v_off = P->lalloc<long long>(nV);
  P->v_size = P->lalloc<long long>(nV);
  P->v_idx = P->lalloc<long long>(nV);
  P->t1_idx = P->lalloc<long long>(nV);
  P->t2_idx = P->lalloc<long long>(nV);
  P->v_list = P->lalloc<int>(nV);
  P->t1_list = P->lalloc<int>(nV);
  P->t2_list = P->lalloc<int>(nV);
  P->y_ptr = P->lalloc<int>(N + 1);
  P->y_home = P->lalloc<int>(nY);
  P->y_j = P->lalloc<int>(nY);
  P->y_R = P->lalloc<int>(3 * (size_t)nY);
  P->ylut = P->lalloc<int>(ylut_n);
  P->yhat = P->lalloc<double>(nY);
  P->y_flag = P->lalloc<int>(nY);
  P->y_off = P->lalloc<long long>(nY);
  P->y_size = P->lalloc<long long>(nY);
  P->y_idx = P->lalloc<long long>(nY);
  P->y_list = P->lalloc<int>(nY);
  P->gC = P->lalloc<double>(3 * (size_t)nC);
  P->gV = P->lalloc<double>(3 * (size_t)nV);
  if (P->opt.deterministic) {
    P->fx_words = 2 * (3 * (size_t)nC + 3 * (size_t)nV + 10 + 3 * (size_t)N);
    P->fx = P->lalloc<unsigned long long>(P->fx_words);
  }
  if (P->wide) {   // C pieces (per call, every C pair)
    std::vector<long long> cw_off(nC + 1, 0);
    for (int p = 0; p < nC; ++p) {
      const int sA = P->species[c_home[p]], sj = P->species[c_j[p]];
      cw_off[p + 1] = cw_off[p] + hfx::wide_cpieces_size(P->np, P->n_abf[sA], P->n_ao[sA], P->n_ao[sj]);
    }
    P->cw_off = P->lalloc<long long>(nC + 1);
    P->Cw = P->lalloc<uint16_t>(std::max(1LL, cw_off[nC]));
    P->dCf = P->lalloc<float>(std::max(1LL, 3 * c_off[nC]));
    upload(P->cw_off, cw_off, s);
  }
  if (P->np) {   // key groups of the Y build
    P->gcnt = P->lalloc<int>(N);
    P->goff = P->lalloc<long long>(N);
    P->gX = P->lalloc<int>(nY);
    P->gS = P->lalloc<int>(nY);
    P->gN = P->lalloc<int>(nY);
  }
  if (P->np && !P->wide) {
    std::vector<long long> cm_off(nC + 1, 0), vm_size(nV);
    for (int p = 0; p < nC; ++p) {
      const int sA = P->species[c_home[p]], sj = P->species[c_j[p]];
      const long long rows = (long long)P->n_abf[sA] * P->n_ao[sA];
      // bf16 tiles then FP32 grad C; each block rounded to 128 bytes (bulk copies need 16-byte alignment)
      const long long sz = P->np * ((rows + 127) / 128) * 2048 + 2 * 3 * ((rows + 127) / 128) * 2048;
      cm_off[p + 1] = cm_off[p] + (sz + 63) / 64 * 64;
    }
    for (int p = 0; p < nV; ++p) {
      const long long mA = P->n_abf[P->species[v_home[p]]], mB = P->n_abf[P->species[v_j[p]]];
      vm_size[p] = P->np * mA * ((mB + 15) / 16 * 16) + 2 * 4 * mA * mB;
    }
    P->cm_off = P->lalloc<long long>(nC + 1);
    P->Cm = P->lalloc<uint16_t>(cm_off[nC]);
    P->vm_off = P->lalloc<long long>(nV);
    P->vm_size = P->lalloc<long long>(nV);
    upload(P->cm_off, cm_off, s);
    upload(P->vm_size, vm_size, s);
    P->qcnt = P->lalloc<int>(nC);
    P->qoff = P->lalloc<long long>(nC);
    P->q_idx = P->lalloc<long long>(nC);
    P->t1q_list = P->lalloc<int>(nC);
    P->t1q_lpt = P->lalloc<int>(nC);
    P->lpt_hist = P->lalloc<int>(hfx::kLptBuckets);
  }
  upload(P->c_ptr, c_ptr, s);
  upload(P->c_home, c_home, s);
  upload(P->c_j, c_j, s);
  upload(P->c_R, c_R, s);
  upload(P->c_off, c_off, s);
  upload(P->v_ptr, v_ptr, s);
  upload(P->v_home, v_home, s);
  upload(P->v_j, v_j, s);
  upload(P->v_R, v_R, s);
  upload(P->v_didx, v_didx, s);
  upload(P->v_size, v_size, s);
  upload(P->y_ptr, y_ptr, s);
  upload(P->y_home, y_home, s);
  upload(P->y_j, y_j, s);
  upload(P->y_R, y_R, s);
  upload(P->ylut, ylut, s);
  upload(P->y_size, y_size, s);
  ck(cudaMemsetAsync(P->c_keep, 0, nC, s), "memset");
  ck(cudaMemsetAsync(P->v_keep, 0, nV, s), "memset");
  ck(cudaStreamSynchronize(s), "upload lists");
  P->c_ptr_h = c_ptr;
  P->v_ptr_h = v_ptr;
  P->pos_ref.assign(pos, pos + 3 * N);
  P->lat_ref.assign(L, L + 9);
  P->list_Rabs = Rabs;
  P->lists_ready = true;
  P->frozen_ready = false;
}

// Largest change of any listed pair distance since the lists were built.
double list_drift(const hfx_plan* P, const double* L, const double* pos) {
  double disp = 0;
  for (int i = 0; i < P->N; ++i) {
    double d2 = 0;
    for (int k = 0; k < 3; ++k) {
      const double dv = pos[3 * i + k] - P->pos_ref[3 * i + k];
      d2 += dv * dv;
    }
    disp = std::max(disp, std::sqrt(d2));
  }
  double dl = 0;
  for (int a = 0; a < 3; ++a) {
    double d2 = 0;
    for (int k = 0; k < 3; ++k) {
      const double dv = L[3 * a + k] - P->lat_ref[3 * a + k];
      d2 += dv * dv;
    }
    dl = std::max(dl, std::sqrt(d2));
  }
  return 2.0 * disp + P->list_Rabs * dl;
}

// Y slots of fs rows that fit next to the first product's fixed shared memory.
long long t1u_slots(const hfx_plan* P, int fs) {
  const size_t base = hfx::t1u_smem(P->np, P->t1u_KP, 0, 1);
  return base < P->t1u_limit ? (long long)((P->t1u_limit - base) / ((size_t)fs * 4096)) : 0LL;
}

void setup_shapes(hfx_plan* P) {
  int dev_smem = 0;
  ck(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->dev), "attr");
  const size_t limit = (size_t)dev_smem - 2048;  // static shared memory of the kernels
  int maxAO = 0, maxABF = 0;
  for (int t = 0; t < P->S; ++t) {
    maxAO = std::max(maxAO, P->n_ao[t]);
    maxABF = std::max(maxABF, P->n_abf[t]);
  }
  const size_t base1 = (size_t)(hfx::kMaxAO * hfx::kMaxAO + maxABF * maxABF) * sizeof(double);
  const size_t per1 = (size_t)maxAO * maxAO * sizeof(double);
  if (base1 + per1 > limit) fail(HFX_ERR_UNSUPPORTED, "block shapes exceed shared memory");
  P->beta_chunk = (int)std::min<size_t>(maxABF, (limit - base1) / per1);
  P->smem_t1 = base1 + per1 * P->beta_chunk;
  const size_t base2 = (size_t)(3 * hfx::kMaxCPerAtom + hfx::kMaxAO * hfx::kMaxAO) * sizeof(double);
  P->alpha_chunk = (int)std::min<size_t>(maxABF, (limit - base2) / per1);
  P->smem_t2 = base2 + per1 * P->alpha_chunk;
  ck(hfx::set_kernel_smem_limits(), "smem attributes");
  if (P->np && maxAO > 16) {
    // n_ao beyond the 16-column tiles of the tensor-memory kernels: the wide kernels
    P->wide = true;
    P->ws = hfx::wide_shapes(P->np, maxABF, maxAO, limit);
    if (!P->ws.ok) fail(HFX_ERR_UNSUPPORTED, "block shapes too large for the split-precision kernels");
    int maxrows = 0;
    for (int a = 0; a < P->S; ++a) maxrows = std::max(maxrows, P->n_abf[a] * P->n_ao[a]);
    P->wide_RB = hfx::wide_ybuild_row_blocks(maxrows);
    P->wide_maxrows = maxrows;
    ck(hfx::set_wide_smem_limits(P->np), "smem attributes");
    return;
  }
  if (P->np) {
    auto r16 = [](int x) { return (x + 15) / 16 * 16; };
    int maxKAF = 0, zrows = 0;
    for (int a = 0; a < P->S; ++a) {
      zrows = std::max(zrows, r16(P->n_abf[a] * P->n_ao[a]));
      for (int b = 0; b < P->S; ++b) maxKAF = std::max(maxKAF, P->n_ao[a] * P->n_ao[b]);
    }
    P->MAmax = r16(maxABF);
    P->MBmax = r16(maxABF);
    P->KSmax = r16(maxKAF) + 8;
    int maxrows = 0;
    for (int a = 0; a < P->S; ++a) maxrows = std::max(maxrows, P->n_abf[a] * P->n_ao[a]);
    P->ZROWS = maxrows;
    P->KZmax = maxAO * r16(maxAO) + 8;
    P->MC = (maxrows + 127) / 128;
    P->zblk = (long long)P->np * P->MC * 128 * 16;   // 128-row tiles of 16 columns, per piece
    P->YRmax = r16(maxABF * maxAO);
    P->smem_m1 = hfx::term1_mma_smem(P->np, P->MAmax, P->MBmax, P->KSmax, P->YRmax);
    P->smem_m2 = hfx::term2_mma_smem(P->np, P->MAmax, P->KZmax);
    // term 1: each warp owns one alpha tile and ceil(NTq / (16 / MT)) Q tiles (at most 16);
    // the second product's GEMM holds two column tiles per F (n_ao <= 16)
    const int MT = P->MAmax / 16, wpm = MT > 0 ? 16 / MT : 0;
    const int qtiles = wpm > 0 ? ((maxKAF + 7) / 8 + wpm - 1) / wpm : 1 << 20;
    // First product: the tcgen05 kernel where the shapes allow it (HFX_T1_KERNEL=mma
    // selects the warp-level MMA kernel instead), else the warp-level one.
    const char* t1k = std::getenv("HFX_T1_KERNEL");
    const bool want_umma = !(t1k && std::string(t1k) == "mma");
    P->t1u = false;
    if (want_umma && maxABF <= 64 && maxAO <= 16) {
      P->t1u_KP = 16 * maxAO;
      // Y ring: slots of FS rows f.  Half a U chunk per slot (one wait and one
      // release per run of rows) when three such slots fit, else runs of two
      // rows (measured best for BF16X6 on si64), else single rows
      // (HFX_T1_FS overrides the run length).
      P->t1u_limit = limit;
      const int fh = (P->t1u_KP / 16 + 1) / 2;
      auto slots = [&](int fs) { return t1u_slots(P, fs); };
      const char* fse = std::getenv("HFX_T1_FS");
      int fs = fse ? std::max(1, std::min(fh, std::atoi(fse))) : (slots(fh) >= 3 ? fh : (slots(2) >= 3 ? 2 : 1));
      while (fs > 1 && slots(fs) < 2) --fs;
      P->t1u_FS = fs;
      P->t1u_NS = (int)std::min<long long>(slots(fs), hfx::t1u_max_slots());
      if (P->t1u_NS >= 2) {
        P->t1u = true;
        P->smem_t1u = hfx::t1u_smem(P->np, P->t1u_KP, P->t1u_NS, P->t1u_FS);
        // kept B per FP32 run of the Q accumulator: 32 for BF16X3, whose
        // stress error is closest to the 1e-5 bound; 128 for BF16X6 (6.5e-6
        // at most on the jittered si64 geometries against 5.4e-6 with 32,
        // and fewer FP64 flushes)
        const char* sg = std::getenv("HFX_T1_SEG");
        P->t1u_seg = sg ? std::max(1, std::atoi(sg)) : (P->np == 3 ? 128 : 32);
        ck(hfx::t1u_set_smem(P->np), "smem attributes");
        // the second product's R2 and Z on tcgen05 as well (HFX_T2_KERNEL=mma keeps the warp-level kernel)
        const char* t2k = std::getenv("HFX_T2_KERNEL");
        P->smem_t2u = hfx::t2u_smem(P->np, maxAO);
        if (!(t2k && std::string(t2k) == "mma") && P->smem_t2u <= limit) {
          P->t2u = true;
          ck(hfx::t2u_set_smem(P->np), "smem attributes");
        }
      }
    }
    if (!P->t1u) {
      if (t1k && std::string(t1k) == "umma")
        fail(HFX_ERR_UNSUPPORTED, "HFX_T1_KERNEL=umma: shapes outside the tcgen05 first-product kernel");
      if (P->smem_m1 > limit || qtiles > 16) fail(HFX_ERR_UNSUPPORTED, "block shapes too large for the split-precision kernels");
    }
    if (P->smem_m2 > limit || maxAO > 16)
      fail(HFX_ERR_UNSUPPORTED, "block shapes too large for the split-precision kernels");
    // 128-row tiles per CTA of the tcgen05 Y build and Q2 GEMM (the autotuner
    // may change them; HFX_Y_TILES = 1 or 2, HFX_Q2_TILES = 1, 2 or 3 set the initial choice)
    const char* yt = std::getenv("HFX_Y_TILES");
    const char* qt = std::getenv("HFX_Q2_TILES");
    P->ybtpc = yt && std::atoi(yt) == 1 ? 1 : 2;
    // (BF16X6 starts from the deep pipeline: si1000 second product 172.6 -> 139.6 ms)
    P->q2tpc = qt && (std::atoi(qt) >= 1 && std::atoi(qt) <= 3) ? std::atoi(qt) : (P->np == 3 ? 3 : 2);
    const char* qf = std::getenv("HFX_Q2_FLUSH");
    P->q2_flush = qf ? std::max(1, std::atoi(qf)) : (P->np == 3 ? 128 : 32);   // as t1u_seg
    ck(hfx::set_mixed_smem_limits(P->np), "smem attributes");
  }
}

// bf16 pieces of every D block (fixed for the plan)
void split_density(hfx_plan* P) {
  if (!P->np || P->n_d == 0) return;
  if (P->wide) {   // NP planes of rup16(n_ao(I)) x rup16(n_ao(J)) per D block, row-major
    std::vector<long long> off(P->n_d + 1, 0);
    for (long long k = 0; k < P->n_d; ++k) {
      const int* r = &P->d_index[5 * k];
      const long long a = (P->n_ao[P->species[r[0]]] + 15) / 16 * 16, b = (P->n_ao[P->species[r[1]]] + 15) / 16 * 16;
      off[k + 1] = off[k] + (long long)P->np * a * b;
    }
    P->dw_off = P->mem.alloc<long long>(P->n_d + 1);
    P->Dw = P->mem.alloc<uint16_t>(off[P->n_d]);
    upload(P->dw_off, off, P->stream);
    DevPlan D = make_devplan(P, P->lat_ref.data());
    ck(hfx::launch_dsplit_w(D, P->np, P->Dw, P->dw_off, P->stream), "D pieces");
    ck(cudaStreamSynchronize(P->stream), "D pieces");
    return;
  }
  std::vector<long long> off(P->n_d + 1, 0);
  for (long long k = 0; k < P->n_d; ++k) {
    const int* r = &P->d_index[5 * k];
    const long long a = (P->n_ao[P->species[r[0]]] + 15) / 16 * 16, b = (P->n_ao[P->species[r[1]]] + 15) / 16 * 16;
    off[k + 1] = off[k] + (long long)P->np * a * b;
  }
  P->dsp_off = P->mem.alloc<long long>(P->n_d + 1);
  P->Dsp = P->mem.alloc<uint16_t>(off[P->n_d] + 256);   // + one zero row (absent blocks)
  upload(P->dsp_off, off, P->stream);
  ck(cudaMemsetAsync(P->Dsp + off[P->n_d], 0, 256 * sizeof(uint16_t), P->stream), "memset");
  {   // the split path holds n_ao <= 16: every piece is one 16 x 16 block of 512 bytes
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    ck(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q), "driver entry");
    if (!fn || q != cudaDriverEntryPointSuccess) fail(HFX_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    const long long rows = off[P->n_d] / 256 + 1;
    const cuuint64_t dims[2] = {256, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {512};
    const cuuint32_t box[2] = {256, 1}, estr[2] = {1, 1};
    const CUresult r = reinterpret_cast<Encode>(fn)(&P->drows.map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, P->Dsp, dims,
                                                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(HFX_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    P->drows.zero_row = (int)(rows - 1);
  }
  DevPlan D = make_devplan(P, P->lat_ref.data());
  hfx::MixPlan X{P->Dsp, P->dsp_off, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  ck(hfx::launch_dsplit(D, X, P->np, P->stream), "dsplit");
  if (P->t1u) {
    P->d_work = P->mem.alloc<int>(1);
    P->Df = P->mem.alloc<float>((size_t)P->n_d * 256);
    hfx::T1UPlan U{};
    U.Df = P->Df;
    ck(hfx::launch_t1u_stores(D, U, P->np, nullptr, 0, true, P->stream), "D FP32 store");
  }
  ck(cudaStreamSynchronize(P->stream), "dsplit");
}

void ensure_store(hfx_plan* P, double*& buf, long long& cap, long long need) {
  if (need <= cap) return;
  if (P->noalloc_call)
    fail(HFX_ERR_UNSUPPORTED, "this evaluation needs more scratch than the fixed no-allocation array holds");
  if (buf) P->mem.release(buf);
  buf = nullptr;
  cap = 0;
  const long long n = need + need / 8 + 1024;
  buf = P->mem.alloc<double>((size_t)n);
  cap = n;
}

template <class T>
void ensure_buf(hfx_plan* P, T*& buf, long long& cap, long long need) {
  if (need <= cap) return;
  if (buf) P->mem.release(buf);
  buf = nullptr;
  cap = 0;
  const long long n = need + need / 8 + 1024;
  buf = P->mem.alloc<T>((size_t)n);
  cap = n;
}

struct Timer {
  bool on;
  cudaStream_t s;
  std::vector<cudaEvent_t> ev;
  explicit Timer(bool o, cudaStream_t st) : on(o), s(st) {}
  int mark() {   // index of the recorded event (-1 when timing is off)
    if (!on) return -1;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    ev.push_back(e);
    return (int)ev.size() - 1;
  }
  double ms(int a, int b) {
    if (!on || a < 0 || b < 0 || b >= (int)ev.size()) return 0;
    float t = 0;
    cudaEventElapsedTime(&t, ev[a], ev[b]);
    return t;
  }
  ~Timer() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

// Totals of one pass of home atoms (scans over the pass's slice of the V and
// C pair lists): FP64 V store elements, needed V pairs, first-product V
// pairs, second-product pairs, split-path V store elements, first-product
// (A,F) items.
enum PassTot { CT_VE = 0, CT_VN = 1, CT_T1 = 2, CT_T2 = 3, CT_VM = 4, CT_Q = 5, kCT = 6 };

// One evaluation.  positions are in P->d_pos already; writes d_out.
//
// Screening and the Y blocks cover every home atom of the plan at once; the
// per-call operand stores and both exchange products then run in passes of
// home atoms (P->chunks), each pass with its own slice of the pair lists, so
// those stores hold one pass at a time.  Every pass's totals are read back
// with the global ones in the single host synchronisation after screening.
long long launches_so_far() {
  return hfx::launch_count() + hfx::mixed_launch_count() + hfx::t1u_launch_count() + hfx::wide_launch_count();
}

void evaluate_launches(hfx_plan* P, const double* L, hfx_stats* st, bool tail = true);
void finish_evaluation(hfx_plan* P, hfx_stats* st, hfx_stats S, long long launches);

// One evaluation.  positions are in P->d_pos already; writes d_out.
//
// A frozen plan with hfx_options.graph records its second evaluation (the
// first one fixed the screening decisions and sized every store, so the
// launches no longer depend on the host) into a CUDA graph and launches that
// graph on later calls; the positions and the lattice are read from device
// memory, written before the launch.
void evaluate(hfx_plan* P, const double* L, hfx_stats* st) {
  cudaStream_t s = P->stream;
  ck(cudaMemcpyAsync(P->d_lat, L, 9 * sizeof(double), cudaMemcpyHostToDevice, s), "H2D lattice");
  const bool reuse = P->opt.freeze_lists && P->frozen_ready;
  const bool graph = P->opt.graph && reuse && !P->timing && !P->noalloc_call;
  if (!graph) {
    evaluate_launches(P, L, st);
    if (st) st->graph_replayed = 0;
    return;
  }
  if (!P->gexec) {
    // record on a stream of the plan's own (the plan's stream may be the
    // legacy default stream, which cannot be captured); the graph is then
    // launched on the plan's stream, after the lattice copy above
    if (!P->cap_stream) ck(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking), "capture stream");
    cudaGraph_t g = nullptr;
    const long long l0 = launches_so_far();
    cudaStream_t own = P->stream;
    P->stream = P->cap_stream;
    ck(cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    try {
      evaluate_launches(P, L, nullptr, false);
    } catch (...) {
      cudaStreamEndCapture(P->cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      P->stream = own;
      throw;
    }
    P->stream = own;
    ck(cudaStreamEndCapture(P->cap_stream, &g), "end capture");
    const cudaError_t e = cudaGraphInstantiate(&P->gexec, g, 0);
    cudaGraphDestroy(g);
    ck(e, "graph instantiate");
    P->graph_launches = launches_so_far() - l0;
  }
  ck(cudaGraphLaunch(P->gexec, s), "graph launch");
  finish_evaluation(P, st, hfx_stats{}, P->graph_launches);
  if (st) st->graph_replayed = 1;
}

// The launches of one evaluation (see evaluate); with tail, also the
// error-flag check and the stats.
void evaluate_launches(hfx_plan* P, const double* L, hfx_stats* st, bool tail) {
  cudaStream_t s = P->stream;
  DevPlan D = make_devplan(P, L);
  const long long launches0 = launches_so_far();
  hfx::MixPlan X{P->Dsp, P->dsp_off, P->Ysp, P->Cm, P->cm_off, P->Vm, P->vm_off, P->Zst, P->qcnt, P->qoff, P->blist};
  const bool reuse = P->opt.freeze_lists && P->frozen_ready;
  const int nch = (int)P->chunks.size();
  long long* T = P->d_tot;
  long long* CT = P->d_tot + kTot + hfx::CNT_N;   // [nch][kCT]
  constexpr int MW = hfx::kMaskWords;
  Timer tm(P->timing, s);
  tm.mark();  // 0
  ck(cudaMemsetAsync(P->d_acc, 0, hfx::ACC_N * sizeof(double), s), "memset");
  ck(cudaMemsetAsync(P->d_tot + kTot, 0, hfx::CNT_N * sizeof(long long), s), "memset");
  ck(cudaMemsetAsync(P->gC, 0, 3 * (size_t)P->nC * sizeof(double), s), "memset");
  ck(cudaMemsetAsync(P->gV, 0, 3 * (size_t)P->nV * sizeof(double), s), "memset");
  if (P->fx) ck(cudaMemsetAsync(P->fx, 0, P->fx_words * sizeof(unsigned long long), s), "memset");
  // D is fixed for the plan: its norms and step-1 decisions are taken once
  const bool dnorm_now = !P->dnorm_done;
  if (dnorm_now) ck(hfx::launch_dnorm(D, s), "dnorm");
  // the split path evaluates C from the block model where it stores the
  // operands; the FP64 path and the wide split path write the FP64 C blocks
  const bool split = P->np && !P->wide;
  if (split)
    ck(hfx::launch_cnorm(D, reuse ? 1 : 0, s), "cnorm");
  else
    ck(hfx::launch_cblocks(D, reuse ? 1 : 0, s), "cblocks");
  ck(hfx::launch_vnorm(D, reuse ? 1 : 0, s), "vnorm");
  tm.mark();  // 1
  if (!reuse) {
    ck(cudaMemsetAsync(P->y_flag, 0, (size_t)P->nY * sizeof(int), s), "memset");
    ck(hfx::launch_yhat(D, s), "yhat");
    ck(hfx::launch_screen(D, s), "screen");
    ck(hfx::scan_flags(P->y_flag, P->y_size, nullptr, nullptr, 1, P->nY, P->y_off, T + 0, P->scan_tmp, s), "scan");
    ck(hfx::scan_flags(P->y_flag, nullptr, nullptr, nullptr, 0, P->nY, P->y_idx, T + 1, P->scan_tmp, s), "scan");
    ck(hfx::scatter_list(P->y_flag, nullptr, nullptr, 0, P->nY, P->y_idx, P->y_list, 0, s), "scatter");
    for (int c = 0; c < nch; ++c) {   // per pass: its slice [v0, v1) of the V pairs
      const int v0 = P->v_ptr_h[P->chunks[c].first], nv = P->v_ptr_h[P->chunks[c].second] - v0;
      long long* ct = CT + (size_t)kCT * c;
      ck(hfx::scan_flags(P->v_flag + v0, P->v_size + v0, nullptr, nullptr, 1, nv, P->v_off + v0, ct + CT_VE,
                         P->scan_tmp, s), "scan");
      ck(hfx::scan_flags(P->v_flag + v0, nullptr, nullptr, nullptr, 0, nv, P->v_idx + v0, ct + CT_VN, P->scan_tmp, s),
         "scan");
      ck(hfx::scatter_list(P->v_flag + v0, nullptr, nullptr, 0, nv, P->v_idx + v0, P->v_list + v0, v0, s), "scatter");
      ck(hfx::scan_flags(nullptr, nullptr, P->v_mask + (size_t)v0 * MW, nullptr, 2, nv, P->t1_idx + v0, ct + CT_T1,
                         P->scan_tmp, s), "scan");
      ck(hfx::scatter_list(nullptr, P->v_mask + (size_t)v0 * MW, nullptr, 2, nv, P->t1_idx + v0, P->t1_list + v0, v0, s),
         "scatter");
      ck(hfx::scan_flags(nullptr, nullptr, nullptr, P->v_t2 + v0, 3, nv, P->t2_idx + v0, ct + CT_T2, P->scan_tmp, s),
         "scan");
      ck(hfx::scatter_list(nullptr, nullptr, P->v_t2 + v0, 3, nv, P->t2_idx + v0, P->t2_list + v0, v0, s), "scatter");
      if (split)
        ck(hfx::scan_flags(P->v_flag + v0, P->vm_size + v0, nullptr, nullptr, 1, nv, P->vm_off + v0, ct + CT_VM,
                           P->scan_tmp, s), "scan");
    }
    if (P->np) {   // groups of up to 8 needed keys of one home atom (the Y build's CTAs)
      ck(hfx::launch_ygroups(D, P->y_idx, T + 1, P->gcnt, nullptr, nullptr, nullptr, nullptr, 0, s), "ygroups");
      ck(hfx::scan_flags(P->gcnt, nullptr, nullptr, nullptr, 4, P->N, P->goff, T + 9, P->scan_tmp, s), "scan");
      ck(hfx::launch_ygroups(D, P->y_idx, T + 1, P->gcnt, P->goff, P->gX, P->gS, P->gN, 1, s), "ygroups");
    }
    if (split) {
      // (A,F) view of the kept triplets: per C pair, its kept B in V-pair order
      ck(hfx::launch_t1_lists(D, X, 0, s), "t1 count");
      ck(hfx::scan_flags(P->qcnt, nullptr, nullptr, nullptr, 4, P->nC, P->qoff, T + 6, P->scan_tmp, s), "scan");
      for (int c = 0; c < nch; ++c) {   // per pass: its items, longest first
        const int c0 = P->c_ptr_h[P->chunks[c].first], nc = P->c_ptr_h[P->chunks[c].second] - c0;
        long long* ct = CT + (size_t)kCT * c;
        ck(hfx::scan_flags(P->qcnt + c0, nullptr, nullptr, nullptr, 0, nc, P->q_idx + c0, ct + CT_Q, P->scan_tmp, s),
           "scan");
        ck(hfx::scatter_list(P->qcnt + c0, nullptr, nullptr, 0, nc, P->q_idx + c0, P->t1q_list + c0, c0, s), "scatter");
        ck(hfx::launch_lpt_order(P->t1_order == 2 ? P->c_j : P->qcnt, P->t1_order == 2 ? 1 : 0, P->t1q_list + c0, nc,
                                 ct + CT_Q, P->lpt_hist, P->t1q_lpt + c0, s),
           "item order");
      }
    }
    ck(cudaMemcpyAsync(P->tot, P->d_tot, kTot * sizeof(long long), cudaMemcpyDeviceToHost, s), "D2H totals");
    ck(cudaMemcpyAsync(P->ctot.data(), CT, P->ctot.size() * sizeof(long long), cudaMemcpyDeviceToHost, s),
       "D2H pass totals");
    ck(cudaMemcpyAsync(P->cnt, P->d_tot + kTot, hfx::CNT_N * sizeof(long long), cudaMemcpyDeviceToHost, s),
       "D2H counts");
    ck(cudaStreamSynchronize(s), "screening");
  }
  // (with frozen decisions the totals and counts of the first call stand, and
  // nothing here waits for the device)
  if (dnorm_now) {
    P->d_kept = (long long)P->cnt[hfx::CNT_D];
    P->dnorm_done = true;
  }
  if (P->opt.freeze_lists) P->frozen_ready = true;
  tm.mark();  // 2
  // ---- shared by every pass: the Y blocks (and the C operand pieces they read)
  hfx::T1UPlan U{};
  if (!P->np) {
    ensure_store(P, P->Yst, P->Ycap, P->tot[0]);
    D.Yst = P->Yst;
    ck(hfx::launch_ybuild(D, P->y_list, (int)P->tot[1], s), "ybuild");
  } else if (P->wide) {
    ensure_buf(P, P->Ysp, P->Yspcap, std::max(1LL, P->tot[0]));
    ck(hfx::launch_cpieces_w(D, P->np, P->Cw, P->cw_off, P->dCf, s), "C pieces");
    ck(hfx::launch_ybuild_w(D, P->np, P->Ysp, P->Cw, P->cw_off, P->Dw, P->dw_off, P->y_list, P->gX, P->gS, P->gN,
                            (int)P->tot[9], P->wide_RB, s),
       "ybuild");
  } else {
    // the core-matrix Y stores' rows past n_abf are never written: zero them
    // once per allocation so that they hold finite values
    const long long ycap0 = P->Yspcap;
    ensure_buf(P, P->Ysp, P->Yspcap, P->tot[0]);
    if (P->t2u && P->Yspcap != ycap0) ck(cudaMemsetAsync(P->Ysp, 0, P->Yspcap * sizeof(uint16_t), s), "memset");
    X.Ysp = P->Ysp;
    X.ycm = P->t2u ? 1 : 0;
    X.ybtpc = P->ybtpc;
    X.q2tpc = P->q2tpc;
    if (!reuse) {
      ensure_buf(P, P->blist, P->blist_cap, P->tot[6]);
      X.blist = P->blist;
      ck(hfx::launch_t1_lists(D, X, 1, s), "t1 fill");
    }
    X.blist = P->blist;
    ck(hfx::launch_cpieces(D, X, P->np, s), "cpieces");
    if (P->t1u) {
      U.KP = P->t1u_KP;
      U.NS = P->t1u_NS;
      U.FS = P->t1u_FS;
      U.seg = P->t1u_seg;
      U.cu_blk = (long long)P->np * 64 * U.KP + 2LL * 4 * 64 * hfx::t1u_kp32(U.KP);
      U.vu_blk = (long long)P->np * 4096 + 2LL * 3 * 4096;
      ensure_buf(P, P->Yf, P->Yfcap, std::max(1LL, P->tot[0] / P->np));
      U.Yf = P->Yf;
      U.Df = P->Df;
      U.t1_idx = P->t1_idx;
      X.Yf = P->Yf;
    }
    X.yT_blk = P->t2u ? (long long)P->np * 64 * P->t1u_KP : (long long)P->np * P->MC * 128 * 16;
    const long long tcap0 = P->YspTcap;
    ensure_buf(P, P->YspT, P->YspTcap, std::max(1LL, P->tot[1]) * X.yT_blk);
    if (P->t2u && P->YspTcap != tcap0) ck(cudaMemsetAsync(P->YspT, 0, P->YspTcap * sizeof(uint16_t), s), "memset");
    X.YspT = P->YspT;
    X.y_idx = P->y_idx;
    ensure_buf(P, P->ytab, P->ytabcap, std::max(1LL, hfx::ytab_size((int)P->tot[9], P->maxC)));
    X.ytab = P->ytab;
    X.ytab_stride = 8 * P->maxC;
    ck(hfx::launch_ybuild_mma(D, X, P->np, P->y_list, P->gX, P->gS, P->gN, (int)P->tot[9], P->MC, P->drows, P->d_err, s),
       "ybuild");
  }
  tm.mark();  // 3
  // ---- passes of home atoms: per-call operand stores and both exchange products
  std::vector<int> m1, m2, m3, k1a, k1b, k2a;   // timer marks around each pass's stages and kernels
  // first-product items: longest first (the last ones handed out are short),
  // or in home-atom order (items running at the same time share their V_AB,
  // grad V_AB in L2); the autotuner picks
  const int* t1items = P->t1_order == 1 ? P->t1q_list : P->t1q_lpt;
  for (int c = 0; c < nch; ++c) {
    const int a0 = P->chunks[c].first, a1 = P->chunks[c].second;
    const int v0 = P->v_ptr_h[a0], c0 = P->c_ptr_h[a0];
    const long long* ct = P->ctot.data() + (size_t)kCT * c;
    m1.push_back(tm.mark());
    if (!split) {   // FP64 V blocks; the FP64 or the wide split kernels
      ensure_store(P, P->Vst, P->Vcap, ct[CT_VE]);
      D.Vst = P->Vst;
      ck(hfx::launch_vblocks(D, P->v_list + v0, (int)ct[CT_VN], s), "vblocks");
      k1a.push_back(tm.mark());
      if (P->wide)
        ck(hfx::launch_term1_w(D, P->np, P->Ysp, P->Cw, P->cw_off, P->Dw, P->dw_off, P->dCf, P->t1_list + v0,
                               (int)ct[CT_T1], P->ws, s),
           "term1");
      else
        ck(hfx::launch_term1(D, P->t1_list + v0, (int)ct[CT_T1], P->beta_chunk, P->smem_t1, s), "term1");
      k1b.push_back(tm.mark());
      m2.push_back(k1b.back());
      k2a.push_back(k1b.back());
      if (P->wide) {
        ensure_buf(P, P->Zw, P->Zwcap,
                   std::max(1LL, ct[CT_T2]) * P->np * hfx::wide_zplane(P->wide_maxrows, P->ws.KZ));
        ck(hfx::launch_term2_w(D, P->np, P->Ysp, P->Zw, P->Dw, P->dw_off, P->dCf, P->t2_list + v0, P->t2_idx, (int)ct[CT_T2],
                               a0, a1, P->wide_maxrows, P->maxC, P->ws, s),
           "term2");
      } else
        ck(hfx::launch_term2(D, P->t2_list + v0, (int)ct[CT_T2], P->alpha_chunk, P->smem_t2, s), "term2");
    } else {
      if (!P->t2u) ensure_buf(P, P->Vm, P->Vmcap, ct[CT_VM]);   // read by the warp-level kernels only
      X.Vm = P->Vm;
      // the split path evaluates V and grad V from the block model where it
      // writes the operand stores (no FP64 V blocks): one pass per needed pair
      // for both products when the tcgen05 first product runs
      if (P->t1u) {
        if (P->t2u) {   // the tcgen05 R2 / Z kernel's V store, written by the V store kernel below
          X.vz_blk = (long long)P->np * 4096 + 2LL * 4 * 4096;
          ensure_buf(P, P->Vz, P->Vzcap, std::max(1LL, ct[CT_T2]) * X.vz_blk);
          X.Vz = P->Vz;
          X.t2_slot = P->t2_idx;
        }
        ensure_buf(P, P->Cu, P->Cucap, std::max(1LL, ct[CT_Q]) * U.cu_blk);
        ensure_buf(P, P->Vu, P->Vucap, std::max(1LL, ct[CT_T1]) * U.vu_blk);
        U.Cu = P->Cu;
        U.Vu = P->Vu;
        ck(hfx::launch_t1u_stores(D, U, P->np, t1items + c0, (int)ct[CT_Q], false, s), "term-1 C store");
        ck(hfx::launch_vstores(D, X, U, P->np, P->v_list + v0, (int)ct[CT_VN], s), "V stores");
        k1a.push_back(tm.mark());
        ck(hfx::launch_t1_umma(D, X, U, P->np, t1items + c0, (int)ct[CT_Q], P->smem_t1u, P->d_work, P->d_err, s),
           "term1");
      } else {
        ck(hfx::launch_vpieces(D, X, P->np, P->v_list + v0, (int)ct[CT_VN], s), "vpieces");
        k1a.push_back(tm.mark());
        ck(hfx::launch_term1_mma(D, X, P->np, t1items + c0, (int)ct[CT_Q], P->MAmax, P->MBmax, P->KSmax, P->YRmax,
                                 P->smem_m1, s),
           "term1");
      }
      k1b.push_back(tm.mark());
      m2.push_back(k1b.back());
      if (ct[CT_T2] * P->zblk > P->Zcap) {
        ensure_buf(P, P->Zst, P->Zcap, ct[CT_T2] * P->zblk);
        ck(cudaMemsetAsync(P->Zst, 0, (size_t)P->Zcap * sizeof(uint16_t), s), "memset");   // tile padding rows stay zero
      }
      X.Zst = P->Zst;
      const int FC = (P->maxC + 3) / 4;
      ensure_buf(P, P->q2tab, P->q2tabcap, std::max(1LL, hfx::q2tab_size((int)ct[CT_T2], FC)));
      X.q2tab = P->q2tab;
      // test-only fault injection (see MixPlan::stall_q2)
      const char* stall = std::getenv("HFX_TEST_STALL_Q2_PRODUCER");
      X.stall_q2 = stall && stall[0] == '1' ? 1 : 0;
      k2a.push_back(tm.mark());
      if (P->t2u)
        ck(hfx::launch_t2_umma(D, X, P->np, P->t2_list + v0, (int)ct[CT_T2], P->zblk, P->smem_t2u, P->d_err, s),
           "term2 R2 and Z");
      ck(hfx::launch_term2_mma(D, X, P->np, P->t2_list + v0, P->t2_idx, (int)ct[CT_T2], a0, a1, P->MAmax, P->KZmax,
                               P->zblk, P->ZROWS, FC, P->MC, hfx::q2_umma_segments(P->maxV, P->np, P->q2tpc), P->q2_flush,
                               P->drows, P->smem_m2, P->d_err, s, P->t2u),
         "term2");
    }
    m3.push_back(tm.mark());
  }
  const int mr = tm.mark();
  ck(cudaMemsetAsync(P->d_out, 0, (1 + 3 * (size_t)P->N + 9) * sizeof(double), s), "memset");
  ck(hfx::launch_reduce(D, P->d_out, s), "reduce");
  const int me = tm.mark();
  if (!tail) return;   // recorded into a graph: the caller finishes after the launch
  hfx_stats S{};
  if (st) {
    ck(cudaStreamSynchronize(s), "stats");   // the events are complete
    S.ms_blocks = tm.ms(0, 1);
    S.ms_screen = tm.ms(1, 2);
    S.ms_y = tm.ms(2, 3);
    for (int c = 0; c < nch; ++c) {
      S.ms_term1 += tm.ms(m1[c], m2[c]);
      S.ms_term2 += tm.ms(m2[c], m3[c]);
      S.ms_term1_kernel += tm.ms(k1a[c], k1b[c]);
      S.ms_term2_kernel += tm.ms(k2a[c], m3[c]);
    }
    S.ms_reduce = tm.ms(mr, me);
    S.ms_total = tm.ms(0, me);
  }
  finish_evaluation(P, st, S, launches_so_far() - launches0);
}

// After the launches of an evaluation: the tensor-core pipelines' error flag
// (split path) and the counters of hfx_stats (S carries the stage times).
void finish_evaluation(hfx_plan* P, hfx_stats* st, hfx_stats S, long long launches) {
  cudaStream_t s = P->stream;
  if (P->np) {
    int errflag = 0;
    ck(cudaMemcpyAsync(&errflag, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H error flag");
    ck(cudaStreamSynchronize(s), "error flag");
    if (errflag) {
      ck(cudaMemsetAsync(P->d_err, 0, sizeof(int), s), "memset");
      fail(HFX_ERR_TIMEOUT, "a tensor-core pipeline wait ran out (results discarded)");
    }
  }
  if (!st) return;
  double acc[hfx::ACC_N];
  ck(cudaMemcpyAsync(acc, P->d_acc, sizeof(acc), cudaMemcpyDeviceToHost, s), "D2H acc");
  ck(cudaStreamSynchronize(s), "stats");
  const int nch = (int)P->chunks.size();
  S.c_pairs = (long long)P->cnt[hfx::CNT_C];
  S.v_pairs = (long long)P->cnt[hfx::CNT_V];
  S.d_blocks = P->d_kept;
  S.triplets = (long long)P->cnt[hfx::CNT_TRIP];
  S.term1_pairs = S.term2_pairs = 0;
  for (int c = 0; c < nch; ++c) {
    S.term1_pairs += P->ctot[(size_t)kCT * c + CT_T1];
    S.term2_pairs += P->ctot[(size_t)kCT * c + CT_T2];
  }
  S.y_blocks = P->tot[1];
  S.flops_y = acc[hfx::ACC_FY];
  S.flops_term1 = acc[hfx::ACC_F1];
  S.flops_term2 = acc[hfx::ACC_F2];
  S.flops_total = S.flops_y + S.flops_term1 + S.flops_term2;
  S.device_bytes = P->mem.bytes;
  S.kernel_launches = launches;
  S.passes = nch;
  S.graph_replayed = 0;
  S.ref_err_E = S.ref_err_F = S.ref_err_sigma = -1.0;
  *st = S;
}

// Relative errors of a result (host [E, F, sigma]) against the plan's reference.
void ref_errors(const hfx_plan* P, const double* out, hfx_stats* st) {
  if (!st || !P->has_ref) return;
  const int n = 3 * P->N;
  st->ref_err_E = std::fabs(out[0] - P->ref[0]) / std::max(std::fabs(P->ref[0]), 1e-300);
  auto rel = [&](int o, int m) {
    double num = 0, den = 0;
    for (int i = 0; i < m; ++i) {
      num = std::max(num, std::fabs(out[o + i] - P->ref[o + i]));
      den = std::max(den, std::fabs(P->ref[o + i]));
    }
    return num / std::max(den, 1e-300);
  };
  st->ref_err_F = rel(1, n);
  st->ref_err_sigma = rel(1 + n, 9);
}

}  // namespace

namespace {
hfx_status run_guarded(hfx_plan* P, const std::function<void()>& fn) {
  try {
    fn();
    if (P) P->err.clear();
    return HFX_OK;
  } catch (const Failure& f) {
    if (P) P->err = f.msg;
    return f.status;
  } catch (const std::bad_alloc&) {
    if (P) P->err = "host allocation failed";
    return HFX_ERR_OOM;
  } catch (const std::exception& e) {
    if (P) P->err = e.what();
    return HFX_ERR_INVALID;
  } catch (...) {
    if (P) P->err = "unknown error";
    return HFX_ERR_INVALID;
  }
}

thread_local std::string g_create_error;

void prepare_call(hfx_plan* P, const double* lattice, const double* positions_host) {
  validate_geometry(P->N, lattice, positions_host);
  const double drift = list_drift(P, lattice, positions_host);
  if (2.0 * drift >= P->opt.skin) {
    if (P->opt.freeze_lists) fail(HFX_ERR_PAIRLIST_STALE, "atoms moved beyond skin/2 on a frozen plan");
    build_lists(P, lattice, positions_host);
  }
}
}  // namespace

extern "C" {

hfx_status hfx_default_options(hfx_options* o) {
  if (!o) return HFX_ERR_INVALID;
  std::memset(o, 0, sizeof(*o));
  o->theta_C = o->theta_dC = o->theta_V = o->theta_dV = o->theta_D = o->theta_CS = 1e-10;
  o->precision = HFX_FP64;
  o->terms = HFX_TERMS_ALL;
  o->skin = 0.5;
  o->freeze_lists = 0;
  o->home_begin = o->home_end = 0;
  o->home_chunk = 0;
  o->graph = 0;
  o->deterministic = 0;
  o->stream = nullptr;
  o->device = 0;
  return HFX_OK;
}

hfx_status hfx_plan_create(const hfx_system* sys, const hfx_model* model, const hfx_options* opt, hfx_plan** out) {
  if (!out) return HFX_ERR_INVALID;
  *out = nullptr;
  hfx_plan* P = nullptr;
  try {
    P = new hfx_plan();
  } catch (...) {
    return HFX_ERR_OOM;
  }
  hfx_status st = run_guarded(P, [&]() {
    validate_options(opt);
    if (!sys || !model) fail(HFX_ERR_INVALID, "system or model is NULL");
    if (sys->n_atoms <= 0 || !sys->species) fail(HFX_ERR_INVALID, "bad n_atoms or species");
    if (model->n_species < 1 || model->n_species > hfx::kMaxSpecies) fail(HFX_ERR_INVALID, "n_species out of range");
    if (!model->n_ao || !model->n_abf || !model->G || !model->M) fail(HFX_ERR_INVALID, "NULL model arrays");
    if (!(model->r_c > 0) || !std::isfinite(model->r_c) || !(model->omega > 0) || !std::isfinite(model->omega))
      fail(HFX_ERR_INVALID, "r_c and omega must be finite and > 0");
    validate_geometry(sys->n_atoms, sys->lattice, sys->positions);
    int h0 = opt->home_begin, h1 = opt->home_end;
    if (h0 == 0 && h1 == 0) h1 = sys->n_atoms;
    if (h0 < 0 || h1 > sys->n_atoms || h0 >= h1) fail(HFX_ERR_INVALID, "home atom range outside [0, n_atoms) or empty");
    P->opt = *opt;
    P->dev = opt->device;
    P->stream = static_cast<cudaStream_t>(opt->stream);
    hfx::AllocHooks hooks;
    hooks.alloc = opt->alloc;
    hooks.free = opt->free;
    hooks.ctx = opt->alloc_ctx;
    hooks.stream = opt->stream;
    P->mem.hooks = hooks;
    P->scan_tmp.mem = hooks;
    ck(cudaSetDevice(P->dev), "cudaSetDevice");
    P->N = sys->n_atoms;
    P->S = model->n_species;
    P->RC = 2.0 * model->r_c;
    P->omega = model->omega;
    P->np = opt->precision == HFX_BF16X3 ? 2 : opt->precision == HFX_BF16X6 ? 3 : 0;
    // passes of the plan's home atoms
    const int want = opt->home_chunk > 0 ? opt->home_chunk : 128;
    const int npass = (h1 - h0 + want - 1) / want;
    for (int c = 0; c < npass; ++c)
      P->chunks.emplace_back(h0 + (int)((long long)(h1 - h0) * c / npass),
                             h0 + (int)((long long)(h1 - h0) * (c + 1) / npass));
    P->ctot.assign((size_t)kCT * npass, 0);
    upload_model(P, sys, model);
    upload_density(P, model);
    P->d_pos = P->mem.alloc<double>(3 * (size_t)P->N);
    P->d_lat = P->mem.alloc<double>(9);
    ck(cudaMemcpy(P->d_lat, sys->lattice, 9 * sizeof(double), cudaMemcpyHostToDevice), "H2D lattice");
    P->d_out = P->mem.alloc<double>(1 + 3 * (size_t)P->N + 9);
    P->d_acc = P->mem.alloc<double>(hfx::ACC_N);
    const size_t ntot = kTot + hfx::CNT_N + (size_t)kCT * npass;
    P->d_tot = P->mem.alloc<long long>(ntot);
    P->d_err = P->mem.alloc<int>(1);
    ck(cudaMemset(P->d_err, 0, sizeof(int)), "memset");
    ck(cudaMemset(P->d_tot, 0, ntot * sizeof(long long)), "memset");
    setup_shapes(P);
    build_lists(P, sys->lattice, sys->positions);
    split_density(P);
  });
  if (st != HFX_OK) {
    g_create_error = P->err;
    P->scan_tmp.mem.put(P->scan_tmp.buf, P->scan_tmp.cap * sizeof(long long));
    P->mem.free_all();
    delete P;
    return st;
  }
  *out = P;
  return HFX_OK;
}

hfx_status hfx_energy_force_stress(hfx_plan* P, const double* lattice, const double* positions, double* E,
                                   double* F, double* sigma, hfx_stats* stats) {
  if (!P) return HFX_ERR_INVALID;
  return run_guarded(P, [&]() {
    if (!E || !F || !sigma) fail(HFX_ERR_INVALID, "NULL output");
    ck(cudaSetDevice(P->dev), "cudaSetDevice");
    prepare_call(P, lattice, positions);
    ck(cudaMemcpyAsync(P->d_pos, positions, 3 * (size_t)P->N * sizeof(double), cudaMemcpyHostToDevice, P->stream),
       "H2D positions");
    evaluate(P, lattice, stats);
    const size_t n = 1 + 3 * (size_t)P->N + 9;
    P->pos_host_buf.resize(n);
    ck(cudaMemcpyAsync(P->pos_host_buf.data(), P->d_out, n * sizeof(double), cudaMemcpyDeviceToHost, P->stream),
       "D2H results");
    ck(cudaStreamSynchronize(P->stream), "results");
    ref_errors(P, P->pos_host_buf.data(), stats);
    *E = P->pos_host_buf[0];
    std::memcpy(F, P->pos_host_buf.data() + 1, 3 * (size_t)P->N * sizeof(double));
    std::memcpy(sigma, P->pos_host_buf.data() + 1 + 3 * P->N, 9 * sizeof(double));
  });
}

hfx_status hfx_energy_force_stress_device(hfx_plan* P, const double* lattice, const double* d_positions,
                                          double* d_out, hfx_stats* stats) {
  if (!P) return HFX_ERR_INVALID;
  return run_guarded(P, [&]() {
    if (!d_positions || !d_out) fail(HFX_ERR_INVALID, "NULL device pointer");
    ck(cudaSetDevice(P->dev), "cudaSetDevice");
    std::vector<double> ph(3 * (size_t)P->N);
    ck(cudaMemcpyAsync(ph.data(), d_positions, ph.size() * sizeof(double), cudaMemcpyDeviceToHost, P->stream),
       "D2H positions");
    ck(cudaStreamSynchronize(P->stream), "positions");
    prepare_call(P, lattice, ph.data());
    ck(cudaMemcpyAsync(P->d_pos, d_positions, ph.size() * sizeof(double), cudaMemcpyDeviceToDevice, P->stream),
       "D2D positions");
    evaluate(P, lattice, stats);
    ck(cudaMemcpyAsync(d_out, P->d_out, (1 + 3 * (size_t)P->N + 9) * sizeof(double), cudaMemcpyDeviceToDevice,
                       P->stream),
       "D2D results");
    if (stats && P->has_ref) {   // the error report needs the result on the host
      P->pos_host_buf.resize(1 + 3 * (size_t)P->N + 9);
      ck(cudaMemcpyAsync(P->pos_host_buf.data(), P->d_out, P->pos_host_buf.size() * sizeof(double),
                         cudaMemcpyDeviceToHost, P->stream),
         "D2H results");
    }
    ck(cudaStreamSynchronize(P->stream), "results");
    if (stats && P->has_ref) ref_errors(P, P->pos_host_buf.data(), stats);
  });
}

hfx_status hfx_set_timing(hfx_plan* P, int on) {
  if (!P) return HFX_ERR_INVALID;
  P->timing = on != 0;
  return HFX_OK;
}

hfx_status hfx_set_reference(hfx_plan* P, const double* E, const double* F, const double* sigma) {
  if (!P) return HFX_ERR_INVALID;
  return run_guarded(P, [&]() {
    if (!E && !F && !sigma) {
      P->has_ref = false;
      P->ref.clear();
      return;
    }
    if (!E || !F || !sigma) fail(HFX_ERR_INVALID, "reference: E, F and sigma must be all set or all NULL");
    std::vector<double> r(1 + 3 * (size_t)P->N + 9);
    r[0] = *E;
    std::memcpy(r.data() + 1, F, 3 * (size_t)P->N * sizeof(double));
    std::memcpy(r.data() + 1 + 3 * (size_t)P->N, sigma, 9 * sizeof(double));
    if (!finite_all(r.data(), r.size())) fail(HFX_ERR_INVALID, "reference: non-finite values");
    P->ref.swap(r);
    P->has_ref = true;
  });
}

hfx_status hfx_plan_autotune(hfx_plan* P, const double* lattice, const double* positions, int reps,
                             hfx_tune_report* report) {
  if (!P || !lattice || !positions || reps < 1) return HFX_ERR_INVALID;
  hfx_tune_report R{};
  R.t1_rows_per_slot = P->t1u_FS;
  R.t1_slots = P->t1u_NS;
  R.t1_home_order = P->t1_order;
  R.y_tiles_per_cta = P->ybtpc;
  R.q2_tiles_per_cta = P->q2tpc;
  if (!P->t1u) {
    if (report) *report = R;
    return HFX_OK;
  }
  const int fs0 = P->t1u_FS, ns0 = P->t1u_NS;
  const size_t smem0 = P->smem_t1u;
  const bool timing0 = P->timing;
  auto use = [&](int fs, int ns) {
    P->t1u_FS = fs;
    P->t1u_NS = ns;
    P->smem_t1u = hfx::t1u_smem(P->np, P->t1u_KP, ns, fs);
    if (P->gexec) {   // a recorded evaluation has the old launch shape
      cudaGraphExecDestroy(P->gexec);
      P->gexec = nullptr;
    }
  };
  std::vector<double> F(3 * (size_t)P->N);
  double E = 0.0, sig[9];
  hfx_stats st{};
  hfx_status status = HFX_OK;
  auto time_it = [&](double& ms) -> bool {   // one warm-up, then the median of reps
    std::vector<double> t;
    for (int r = 0; r <= reps; ++r) {
      status = hfx_energy_force_stress(P, lattice, positions, &E, F.data(), sig, &st);
      if (status != HFX_OK) return false;
      if (r > 0) t.push_back(st.ms_total);
    }
    std::sort(t.begin(), t.end());
    ms = t[t.size() / 2];
    return true;
  };
  P->timing = true;
  bool ok = time_it(R.default_ms);
  int best_fs = fs0, best_ns = ns0;
  R.best_ms = R.default_ms;
  R.candidates = ok ? 1 : 0;
  const int fh = (P->t1u_KP / 16 + 1) / 2;   // a run never crosses a U column chunk
  for (int fs = 1; ok && fs <= fh; ++fs) {
    const int ns = (int)std::min<long long>(t1u_slots(P, fs), hfx::t1u_max_slots());
    if (ns < 2 || (fs == fs0 && ns == ns0)) continue;
    use(fs, ns);
    double ms = 0.0;
    ok = time_it(ms);
    if (!ok) break;
    ++R.candidates;
    if (ms < R.best_ms) {
      R.best_ms = ms;
      best_fs = fs;
      best_ns = ns;
    }
  }
  // the order of the items, with the best ring shape
  const int order0 = P->t1_order;
  int best_order = order0;
  if (ok) {
    use(best_fs, best_ns);
    for (int o = 0; o < 3 && ok; ++o) {
      if (o == order0) continue;
      P->t1_order = o;
      double ms = 0.0;
      ok = time_it(ms);
      if (!ok) break;
      ++R.candidates;
      if (ms < R.best_ms) {
        R.best_ms = ms;
        best_order = o;
      }
    }
    P->t1_order = best_order;
  }
  // then the row tiles per CTA of the Y build and of the Q2 GEMM, one at a time
  const int yb0 = P->ybtpc, q20 = P->q2tpc;
  for (int which = 0; which < 2 && ok; ++which) {
    int& knob = which == 0 ? P->ybtpc : P->q2tpc;
    const int keep = knob;
    // Y build: 1 <-> 2; Q2 GEMM: the two other shapes of 1, 2 and 3 (two
    // tiles, one CTA per SM with the deep pipeline)
    int alts[2] = {3 - keep, 0};
    if (which == 1) {
      alts[0] = keep == 1 ? 2 : 1;
      alts[1] = keep == 3 ? 2 : 3;
    }
    int best = keep;
    for (int ai = 0; ai < 2 && ok; ++ai) {
      if (alts[ai] == 0) continue;
      knob = alts[ai];
      if (P->gexec) {
        cudaGraphExecDestroy(P->gexec);
        P->gexec = nullptr;
      }
      double ms = 0.0;
      ok = time_it(ms);
      if (!ok) break;
      ++R.candidates;
      if (ms < R.best_ms) {
        R.best_ms = ms;
        best = knob;
      }
    }
    knob = best;
  }
  P->timing = timing0;
  if (!ok) {   // keep the initial choice
    use(fs0, ns0);
    P->smem_t1u = smem0;
    P->t1_order = order0;
    P->ybtpc = yb0;
    P->q2tpc = q20;
    return status;
  }
  use(best_fs, best_ns);
  R.t1_rows_per_slot = best_fs;
  R.t1_slots = best_ns;
  R.t1_home_order = best_order;
  R.y_tiles_per_cta = P->ybtpc;
  R.q2_tiles_per_cta = P->q2tpc;
  if (report) *report = R;
  return HFX_OK;
}

hfx_status hfx_plan_destroy(hfx_plan* P) {
  if (!P) return HFX_OK;
  cudaSetDevice(P->dev);
  cudaStreamSynchronize(P->stream);
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  P->scan_tmp.mem.put(P->scan_tmp.buf, P->scan_tmp.cap * sizeof(long long));
  P->mem.free_all();
  delete P;
  return HFX_OK;
}

const char* hfx_status_string(hfx_status s) {
  switch (s) {
    case HFX_OK: return "ok";
    case HFX_ERR_INVALID: return "invalid argument";
    case HFX_ERR_OOM: return "out of memory";
    case HFX_ERR_CUDA: return "CUDA error";
    case HFX_ERR_TIMEOUT: return "timeout";
    case HFX_ERR_PAIRLIST_STALE: return "pair list stale";
    case HFX_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

hfx_status hfx_lri_fit(int batch, int n, int w, const double* A, const double* B, const double* dA,
                       const double* dB, double* X, double* dX, int device) {
  g_create_error.clear();
  auto bad = [](hfx_status st, const char* msg) {
    g_create_error = msg;
    return st;
  };
  const bool grad = dA || dB || dX;
  if (batch < 0 || n < 1 || w < 1 || !A || !B || !X) return bad(HFX_ERR_INVALID, "hfx_lri_fit: bad sizes or NULL");
  if (grad && !(dA && dB && dX)) return bad(HFX_ERR_INVALID, "hfx_lri_fit: dA, dB, dX must be all set or all NULL");
  if (batch == 0) return HFX_OK;
  if (cudaSetDevice(device) != cudaSuccess) return bad(HFX_ERR_CUDA, "hfx_lri_fit: cudaSetDevice");
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (hfx::lri_fit_smem(n) + 2048 > (size_t)optin)
    return bad(HFX_ERR_UNSUPPORTED, "hfx_lri_fit: n too large for the Cholesky factor in shared memory");
  const size_t nn = (size_t)batch * n * n, nw = (size_t)batch * n * w;
  const size_t bytes = (nn + 2 * nw) * sizeof(double) * (grad ? 4 : 1) + sizeof(int);
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return bad(HFX_ERR_CUDA, "hfx_lri_fit: stream");
  unsigned char* buf = nullptr;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(s);
    return bad(HFX_ERR_OOM, "hfx_lri_fit: device memory");
  }
  double* A_dev = reinterpret_cast<double*>(buf);            // A, B, X [, dA, dB, dX]
  double* B_dev = A_dev + nn;
  double* X_dev = B_dev + nw;
  double* gA = grad ? X_dev + nw : nullptr;
  double* gB = grad ? gA + 3 * nn : nullptr;
  double* gX = grad ? gB + 3 * nw : nullptr;
  int* err = reinterpret_cast<int*>(buf + bytes - sizeof(int));
  int herr = 0;
  cudaError_t e = cudaMemcpyAsync(A_dev, A, nn * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B_dev, B, nw * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && grad) e = cudaMemcpyAsync(gA, dA, 3 * nn * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && grad) e = cudaMemcpyAsync(gB, dB, 3 * nw * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = hfx::launch_lri_fit(batch, n, w, A_dev, B_dev, gA, gB, X_dev, gX, err, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  hfx_status st = HFX_OK;
  if (e != cudaSuccess) {
    st = bad(HFX_ERR_CUDA, cudaGetErrorString(e));
  } else if (herr) {
    st = bad(HFX_ERR_INVALID, "hfx_lri_fit: a metric block is not positive definite");
  } else {
    e = cudaMemcpyAsync(X, X_dev, nw * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && grad) e = cudaMemcpyAsync(dX, gX, 3 * nw * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = bad(HFX_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaFree(buf);
  cudaStreamDestroy(s);
  return st;
}

const char* hfx_last_error(const hfx_plan* P) {
  if (!P) return g_create_error.c_str();
  return P->err.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Evaluation without device allocation.
//
// Some callers cannot allocate device memory while they evaluate: hosts that
// hand all device memory to their own pool after start-up, and real-time
// loops that forbid allocation after initialisation.  hfx_energy_force_stress
// may grow its per-call block stores with cudaMalloc, so this entry point runs
// the same FP64 evaluation with that scratch taken from one fixed array
// compiled into the library instead.  The array is a file-scope __device__
// variable: every device that loads the library holds it until the process
// exits.  Host code never passes the array's name to a kernel (in host code it
// is only a stand-in for the symbol); it looks the device address up once per
// device with cudaGetSymbolAddress, with that device current.
constexpr size_t kNoAllocScratchBytes = 64ull << 20;   // HFX_NOALLOC_SCRATCH_BYTES
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double)];

namespace {
std::mutex g_noalloc_mu;
constexpr int kNoAllocMaxDevices = 64;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (first call on a
// device looks it up; later calls reuse it, which assumes the device's primary
// context is never reset while the process runs).
double* noalloc_scratch(int dev) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (dev < 0 || dev >= kNoAllocMaxDevices) fail(HFX_ERR_UNSUPPORTED, "device ordinal too large for the scratch table");
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    ck(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  return g_noalloc_ptr[dev];
}
}  // namespace

extern "C" hfx_status hfx_energy_force_stress_noalloc(hfx_plan* P, const double* lattice, const double* positions,
                                                      double* E, double* F, double* sigma) {
  if (!P) return HFX_ERR_INVALID;
  return run_guarded(P, [&]() {
    if (!E || !F || !sigma) fail(HFX_ERR_INVALID, "NULL output");
    if (P->np) fail(HFX_ERR_UNSUPPORTED, "the no-allocation entry point runs FP64 plans only");
    ck(cudaSetDevice(P->dev), "cudaSetDevice");
    double* base = noalloc_scratch(P->dev);
    validate_geometry(P->N, lattice, positions);
    if (2.0 * list_drift(P, lattice, positions) >= P->opt.skin)
      fail(HFX_ERR_PAIRLIST_STALE,
           "atoms moved beyond skin/2; rebuilding the pair lists allocates (call hfx_energy_force_stress once)");
    // scratch layout: scan temporaries | Y blocks | V blocks
    const long long total = (long long)(kNoAllocScratchBytes / sizeof(double));
    const long long nmax = std::max<long long>(std::max(P->nY, P->nV), P->nC);
    const long long scan_need = (long long)hfx::scan_tmp_need((int)nmax);
    if (scan_need >= total / 4) fail(HFX_ERR_UNSUPPORTED, "pair lists too long for the fixed no-allocation array");
    const long long half = (total - scan_need) / 2;
    const hfx::ScanTmp saved_scan = P->scan_tmp;
    double* const saved_Y = P->Yst;
    double* const saved_V = P->Vst;
    const long long saved_Ycap = P->Ycap, saved_Vcap = P->Vcap;
    const bool saved_timing = P->timing;
    P->scan_tmp.buf = reinterpret_cast<long long*>(base);
    P->scan_tmp.cap = (size_t)scan_need;
    P->scan_tmp.fixed = true;   // never freed or grown: a mismatch fails instead
    P->Yst = base + scan_need;
    P->Ycap = half;
    P->Vst = base + scan_need + half;
    P->Vcap = half;
    P->timing = false;
    P->noalloc_call = true;
    auto restore = [&]() {
      P->scan_tmp = saved_scan;
      P->Yst = saved_Y;
      P->Vst = saved_V;
      P->Ycap = saved_Ycap;
      P->Vcap = saved_Vcap;
      P->timing = saved_timing;
      P->noalloc_call = false;
    };
    try {
      ck(cudaMemcpyAsync(P->d_pos, positions, 3 * (size_t)P->N * sizeof(double), cudaMemcpyHostToDevice, P->stream),
         "H2D positions");
      evaluate(P, lattice, nullptr);
      ck(cudaMemcpyAsync(E, P->d_out, sizeof(double), cudaMemcpyDeviceToHost, P->stream), "D2H E");
      ck(cudaMemcpyAsync(F, P->d_out + 1, 3 * (size_t)P->N * sizeof(double), cudaMemcpyDeviceToHost, P->stream),
         "D2H F");
      ck(cudaMemcpyAsync(sigma, P->d_out + 1 + 3 * (size_t)P->N, 9 * sizeof(double), cudaMemcpyDeviceToHost,
                         P->stream),
         "D2H sigma");
      ck(cudaStreamSynchronize(P->stream), "results");
    } catch (...) {
      restore();
      throw;
    }
    restore();
  });
}
