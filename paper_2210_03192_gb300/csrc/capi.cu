// C ABI of lx3c (declared in include/lx3c.h): basis and plan objects, input
// validation, device-table management and launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lx3c.h"
#include "lx3c_internal.h"

namespace lx3c {
cudaError_t init_constants();
cudaError_t launch_pair_precompute(const DevBasis& orb, const int32_t* pairs, long long npair, int Ka, int Kb,
                                   double* rec, double* ab, cudaStream_t st, int scale_a = 0, int scale_b = 0);
cudaError_t launch_aux_precompute(const DevBasis& aux, const int32_t* auxs, long long naux, int Kc, double* rec,
                                  double* cxyz, cudaStream_t st);
cudaError_t launch_eri3c(const ClassDesc& d, int grid, cudaStream_t st);
cudaError_t launch_boys(const double* T, long long n, int mmax, const double* tab, const double* mid, double cL,
                        double* out, cudaStream_t st);
int eri3c_occupancy(int smem_bytes);
}  // namespace lx3c

using namespace lx3c;

namespace {

thread_local std::string g_err;

lx3c_status fail(lx3c_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

}  // namespace

namespace lx3c {
// lets other translation units report through lx3c_last_error()
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace lx3c

namespace {

#define CUDA_TRY(expr)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) return fail(LX3C_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

// Per-device constant data: Boys tables and uploaded class tables.
struct lx3c::DevState {
  double* boys_tab = nullptr;
  double* boys_mid = nullptr;
  int nsm = 0;
  int smem_per_sm = 0;
  std::map<std::tuple<int, int, int, int>, DevClass> classes;
  // host-buffer path (lx3c_eri3c_host): the two output chunk buffers (grown,
  // never shrunk), the copy stream and its events, made on first use and kept;
  // calls on one device take turns on host_mu
  std::mutex host_mu;
  double* host_buf = nullptr;
  size_t host_cap = 0;  // doubles
  cudaStream_t host_cs = nullptr;
  cudaEvent_t host_done[2] = {}, host_freed[2] = {};
};

namespace {

std::mutex g_mu;
std::map<int, DevState> g_dev;

lx3c_status device_state(DevState** out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  DevState& s = g_dev[dev];
  if (!s.boys_tab) {
    std::vector<double> tab, mid;
    boys_tables(tab, mid);
    CUDA_TRY(cudaMalloc(&s.boys_tab, tab.size() * 8));
    CUDA_TRY(cudaMalloc(&s.boys_mid, mid.size() * 8));
    CUDA_TRY(cudaMemcpy(s.boys_tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(s.boys_mid, mid.data(), mid.size() * 8, cudaMemcpyHostToDevice));
    CUDA_TRY(init_constants());
    CUDA_TRY(cudaDeviceGetAttribute(&s.nsm, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&s.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  }
  *out = &s;
  return LX3C_OK;
}

lx3c_status device_class(DevState* s, const ClassTables& ct, DevClass** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_tuple(ct.la, ct.lb, ct.lc, ct.bra_pure * 2 + ct.hrr2);
  auto it = s->classes.find(key);
  if (it != s->classes.end()) {
    *out = &it->second;
    return LX3C_OK;
  }
  size_t offs[18];
  std::vector<char> blob = class_blob(ct, offs);
  DevClass dc;
  CUDA_TRY(cudaMalloc(&dc.blob, blob.size()));
  CUDA_TRY(cudaMemcpy(dc.blob, blob.data(), blob.size(), cudaMemcpyHostToDevice));
  class_blob_pointers(dc, dc.blob, offs);
  auto r = s->classes.emplace(key, dc);
  *out = &r.first->second;
  return LX3C_OK;
}

}  // namespace

namespace lx3c {

int device_state_get(DevState** out) { return device_state(out); }
int device_class_get(DevState* s, const ClassTables& ct, DevClass** out) { return device_class(s, ct, out); }
const double* dev_boys_tab(const DevState* s) { return s->boys_tab; }
const double* dev_boys_mid(const DevState* s) { return s->boys_mid; }
int dev_nsm(const DevState* s) { return s->nsm; }
int dev_smem(const DevState* s) { return s->smem_per_sm; }

namespace {
template <class T>
size_t append(std::vector<char>& blob, const std::vector<T>& v) {
  size_t off = (blob.size() + 15) & ~size_t(15);
  blob.resize(off + v.size() * sizeof(T) + 16);
  if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}
}  // namespace

std::vector<char> class_blob(const ClassTables& ct, size_t f[18]) {
  std::vector<char> blob;
  f[0] = append(blob, ct.vtab); f[1] = append(blob, ct.wtab); f[2] = append(blob, ct.atab);
  f[3] = append(blob, ct.gptr); f[4] = append(blob, ct.gterm); f[5] = append(blob, ct.gdst);
  f[6] = append(blob, ct.pal); f[7] = append(blob, ct.kptr); f[8] = append(blob, ct.kent);
  f[9] = append(blob, ct.htab); f[10] = append(blob, ct.baptr); f[11] = append(blob, ct.baent);
  f[12] = append(blob, ct.bbptr); f[13] = append(blob, ct.bbent); f[14] = append(blob, ct.gell);
  f[15] = append(blob, ct.gslice); f[16] = append(blob, ct.ktptr); f[17] = append(blob, ct.ktent);
  return blob;
}

void class_blob_pointers(DevClass& dc, const void* dev_blob, const size_t f[18]) {
  const char* b = (const char*)dev_blob;
  dc.vtab = (const uint4*)(b + f[0]);
  dc.wtab = (const int4*)(b + f[1]);
  dc.atab = (const unsigned*)(b + f[2]);
  dc.gptr = (const int*)(b + f[3]);
  dc.gterm = (const unsigned*)(b + f[4]);
  dc.gdst = (const int*)(b + f[5]);
  dc.pal = (const double*)(b + f[6]);
  dc.kptr = (const int*)(b + f[7]);
  dc.kent = (const int2*)(b + f[8]);
  dc.htab = (const uint4*)(b + f[9]);
  dc.baptr = (const int*)(b + f[10]);
  dc.baent = (const int2*)(b + f[11]);
  dc.bbptr = (const int*)(b + f[12]);
  dc.bbent = (const int2*)(b + f[13]);
  dc.gell = (const unsigned*)(b + f[14]);
  dc.gslice = (const int2*)(b + f[15]);
  dc.ktptr = (const int*)(b + f[16]);
  dc.ktent = (const int2*)(b + f[17]);
}

void fill_desc_common(ClassDesc& d, const ClassTables& ct, const DevClass& dc, const double* boys_tab,
                      const double* boys_mid, int orient, int kmax, int Kab_rec, int Kc, const LaunchShape& sh) {
  std::memset(&d, 0, sizeof(d));
  d.la = ct.la; d.lb = ct.lb; d.lc = ct.lc; d.Lab = ct.la + ct.lb; d.L = ct.la + ct.lb + ct.lc;
  d.bra_pure = ct.bra_pure;
  d.ncA = ct.ncA; d.ncB = ct.ncB; d.ncc = ct.ncc;
  d.nA = ct.nA; d.nB = ct.nB; d.nC = ct.nC; d.nblk = d.nA * d.nB * d.nC;
  d.orient = orient;
  d.onA = orient ? ct.nB : ct.nA;
  d.onB = orient ? ct.nA : ct.nB;
  d.Kab = kmax; d.Kc = Kc; d.K = kmax * Kc;
  d.Kab_rec = Kab_rec;
  d.NV = ct.NV; d.NW = ct.NW; d.NF = ct.NF; d.NACC = ct.NACC;
  for (int e = 0; e <= d.Lab; ++e) d.vlev_start[e] = ct.vlev_start[e];
  d.nW = ct.NW;
  d.ngt = ct.nkrow * ct.ncc;
  d.nkrow = ct.nkrow;
  d.nhrr = ct.nhrr;
  for (int j = 0; j <= ct.nhrr; ++j) d.hrows[j] = ct.hrows[j];
  for (int j = 0; j <= ct.nhrr + 1; ++j) d.hstart[j] = ct.hstart[j];
  d.nbA = ct.nbA; d.nbB = ct.nbB;
  d.vtab = dc.vtab; d.wtab = dc.wtab; d.atab = dc.atab; d.gptr = dc.gptr; d.gterm = dc.gterm;
  d.gdst = dc.gdst; d.pal = dc.pal; d.kptr = dc.kptr; d.kent = dc.kent; d.htab = dc.htab;
  d.ktptr = dc.ktptr; d.ktent = dc.ktent;
  d.gell = dc.gell; d.gslice = dc.gslice;
  d.baptr = dc.baptr; d.baent = dc.baent; d.bbptr = dc.bbptr; d.bbent = dc.bbent;
  d.boys_tab = boys_tab; d.boys_mid = boys_mid; d.boys_cL = boys_large_const(d.L);
  d.comp = compensation_bits();
  fill_layout(d, ct, sh);
  d.nchunk = (d.K + d.G - 1) / d.G;
}

int fill_class_desc(ClassDesc& d, const ClassTables& ct, const DevClass& dc, const DevState* ds, int orient,
                    int kmax, int Kab_rec, int Kc, long long naux_for_shape) {
  LaunchShape sh = choose_shape(ct, kmax, Kc, naux_for_shape, ds->smem_per_sm);
  if (sh.smem_bytes < 0 || sh.smem_bytes > 232448) return -1;
  fill_desc_common(d, ct, dc, ds->boys_tab, ds->boys_mid, orient, kmax, Kab_rec, Kc, sh);
  return sh.smem_bytes;
}

}  // namespace lx3c

namespace lx3c {

// Orientation.  HRR (Eq. hrr) builds the target centre's quanta from the
// recurrence centre's through AB; when the target is compact and the
// recurrence centre diffuse, P sits near the target and the transfer
// cancels, amplifying FP64 rounding by about
//   amp = ((|AB| + s) / (|P - target| + s))^l_target,  s = 1/sqrt(2 gamma),
// weighted by the primitive pair's share of the largest prefactor
// |c_a c_b exp(-za zb/gamma AB^2)/gamma| in the pair.  A pair keeps one
// orientation (the one with the smaller worst weighted amp) when that worst
// amp is at most kAmpMax; otherwise every primitive pair runs on its more
// compact centre (two launches, the second accumulating transposed).
// Without HRR (lb = 0) the caller's orientation is always kept.  (Preferring
// the orientation with fewer flops whenever its amp is within kAmpMax saves
// flops only on pairs whose cheaper side amplifies 5-300x, and those pairs
// then miss 1e-12: the smaller amplification wins.)
namespace {
std::atomic<double> g_amp_max{kDefaultAmpMax};
std::atomic<int> g_comp_bits{0};
}  // namespace

double orientation_amp_max() { return g_amp_max.load(); }
int compensation_bits() { return g_comp_bits.load(); }

void split_orientation(const lx3c_basis* orb, int a, int b, int la, int lb, std::vector<int>& primA,
                       std::vector<int>& primB) {
  const double kAmpMax = orientation_amp_max();
  const int Ka = orb->k[a], Kb = orb->k[b];
  const double* A = &orb->xyz[3 * a];
  const double* B = &orb->xyz[3 * b];
  double ab2 = 0;
  for (int x = 0; x < 3; ++x) ab2 += (A[x] - B[x]) * (A[x] - B[x]);
  const double dab = std::sqrt(ab2);
  std::vector<double> wgt(Ka * Kb), ampA(Ka * Kb), ampB(Ka * Kb);
  double wmax = 0;
  for (int ia = 0; ia < Ka; ++ia)
    for (int ib = 0; ib < Kb; ++ib) {
      double za = orb->exps[orb->off[a] + ia], zb = orb->exps[orb->off[b] + ib], g = za + zb;
      double w = std::fabs(orb->coefs[orb->off[a] + ia] * orb->coefs[orb->off[b] + ib]) *
                 std::exp(-za * zb / g * ab2) / g;
      double sg = 1.0 / std::sqrt(2.0 * g);
      ampA[ia * Kb + ib] = std::pow((dab + sg) / (za / g * dab + sg), lb);
      ampB[ia * Kb + ib] = std::pow((dab + sg) / (zb / g * dab + sg), la);
      wgt[ia * Kb + ib] = w;
      wmax = std::max(wmax, w);
    }
  double worstA = 0, worstB = 0;
  for (int r = 0; r < Ka * Kb; ++r) {
    double f = wmax > 0 ? wgt[r] / wmax : 1.0;
    worstA = std::max(worstA, ampA[r] * f);
    worstB = std::max(worstB, ampB[r] * f);
  }
  // one orientation for the whole pair when one is within the threshold:
  // the one with the smaller amplification
  int whole = -1;
  if (lb == 0) whole = 0;
  else if (std::min(worstA, worstB) <= kAmpMax) whole = worstB < worstA ? 1 : 0;
  for (int ia = 0; ia < Ka; ++ia)
    for (int ib = 0; ib < Kb; ++ib) {
      const bool onB = whole >= 0 ? whole == 1 : orb->exps[orb->off[b] + ib] > orb->exps[orb->off[a] + ia];
      (onB ? primB : primA).push_back(ia * Kb + ib);
    }
}

}  // namespace lx3c

// One kernel launch of a plan: one orientation of the pair list.
struct Launch {
  ClassDesc desc;
  int grid = 1;
  long long nsub = 0;
  int4* d_sub = nullptr;
  int* d_prim = nullptr;
  std::vector<int> sub_pair;  // pair index of each sub-pair (ascending)
};

struct lx3c_plan {
  const lx3c_basis* orb = nullptr;
  const lx3c_basis* aux = nullptr;
  int la = 0, lb = 0, lc = 0, bra_pure = 1;
  int Ka = 1, Kb = 1, Kc = 1;
  long long npair = 0, naux = 0;
  int64_t nblk = 0;
  double flops = 0;  // algorithmic flops of one execute, orientation by orientation
  Launch L[2];
  int32_t* d_pairs = nullptr;
  int32_t* d_auxs = nullptr;
  double* d_pairrec = nullptr;
  double* d_pairab = nullptr;
  double* d_auxrec = nullptr;
  double* d_auxc = nullptr;
};

extern "C" {

const char* lx3c_last_error(void) { return g_err.c_str(); }

const char* lx3c_version(void) { return "lx3c 0.1 (sm_103a, FP64)"; }

void lx3c_basis_destroy(lx3c_basis* b) {
  if (!b) return;
  cudaFree(b->d_l);
  cudaFree(b->d_k);
  cudaFree(b->d_off);
  cudaFree(b->d_xyz);
  cudaFree(b->d_exps);
  cudaFree(b->d_coefs);
  delete b;
}

lx3c_status lx3c_basis_create(lx3c_basis** out, int64_t nshell, const int32_t* l, const int32_t* k,
                              const double* xyz, const int32_t* atom, const double* exps, const double* coefs,
                              void* stream) {
  if (!out) return fail(LX3C_EINVAL, "basis_create: null output pointer");
  *out = nullptr;
  if (nshell < 0) return fail(LX3C_EINVAL, "basis_create: negative shell count");
  if (nshell > 0 && (!l || !k || !xyz || !exps || !coefs)) return fail(LX3C_EINVAL, "basis_create: null array");
  std::unique_ptr<lx3c_basis> b(new lx3c_basis);
  b->nshell = nshell;
  b->l.assign(l, l + nshell);
  b->k.assign(k, k + nshell);
  b->off.resize(nshell);
  b->atom.assign(nshell, -1);
  if (atom) b->atom.assign(atom, atom + nshell);
  int64_t np = 0;
  for (int64_t s = 0; s < nshell; ++s) {
    if (l[s] < 0 || l[s] > std::max(LX3C_LMAX_ORB, LX3C_LMAX_AUX))
      return fail(LX3C_ENOTSUP, "basis_create: shell " + std::to_string(s) + " has unsupported l");
    if (k[s] < 1 || k[s] > LX3C_KMAX)
      return fail(LX3C_ENOTSUP, "basis_create: shell " + std::to_string(s) + " has unsupported K");
    b->off[s] = np;
    np += k[s];
  }
  b->nprim = np;
  b->xyz.assign(xyz, xyz + 3 * nshell);
  b->exps.assign(exps, exps + np);
  b->coefs.assign(coefs, coefs + np);
  for (int64_t i = 0; i < 3 * nshell; ++i)
    if (!std::isfinite(b->xyz[i])) return fail(LX3C_EINVAL, "basis_create: non-finite centre");
  for (int64_t i = 0; i < np; ++i) {
    if (!(b->exps[i] > 0.0) || !std::isfinite(b->exps[i]))
      return fail(LX3C_EINVAL, "basis_create: exponent must be finite and > 0");
    if (!std::isfinite(b->coefs[i])) return fail(LX3C_EINVAL, "basis_create: non-finite coefficient");
  }
  lx3c_status rc = basis_upload(b.get(), (cudaStream_t)stream);
  if (rc) return rc;
  *out = b.release();
  return LX3C_OK;
}

}  // extern "C"

namespace lx3c {

lx3c_status basis_upload(lx3c_basis* b, cudaStream_t st) {
  const int64_t nshell = b->nshell, np = b->nprim;
  size_t n = (size_t)std::max<int64_t>(nshell, 1), npp = (size_t)std::max<int64_t>(np, 1);
  CUDA_TRY(cudaMalloc(&b->d_l, n * 4));
  CUDA_TRY(cudaMalloc(&b->d_k, n * 4));
  CUDA_TRY(cudaMalloc(&b->d_off, n * 8));
  CUDA_TRY(cudaMalloc(&b->d_xyz, n * 24));
  CUDA_TRY(cudaMalloc(&b->d_exps, npp * 8));
  CUDA_TRY(cudaMalloc(&b->d_coefs, npp * 8));
  if (nshell > 0) {
    CUDA_TRY(cudaMemcpyAsync(b->d_l, b->l.data(), nshell * 4, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(b->d_k, b->k.data(), nshell * 4, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(b->d_off, b->off.data(), nshell * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(b->d_xyz, b->xyz.data(), nshell * 24, cudaMemcpyHostToDevice, st));
  }
  if (np > 0) {
    CUDA_TRY(cudaMemcpyAsync(b->d_exps, b->exps.data(), np * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(b->d_coefs, b->coefs.data(), np * 8, cudaMemcpyHostToDevice, st));
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  return LX3C_OK;
}

}  // namespace lx3c

extern "C" {

void lx3c_plan_destroy(lx3c_plan* p) {
  if (!p) return;
  cudaFree(p->d_pairs);
  cudaFree(p->d_auxs);
  cudaFree(p->d_pairrec);
  cudaFree(p->d_pairab);
  cudaFree(p->d_auxrec);
  cudaFree(p->d_auxc);
  for (auto& l : p->L) {
    cudaFree(l.d_sub);
    cudaFree(l.d_prim);
  }
  delete p;
}

namespace {

// Fill one launch descriptor for class (l1, l2 | lc) over a sub-pair list.
lx3c_status make_launch(DevState* ds, lx3c_plan* p, int orient, const std::vector<int4>& sub,
                        const std::vector<int>& prim, int kmax, cudaStream_t st) {
  Launch& L = p->L[orient];
  L.nsub = (long long)sub.size();
  if (L.nsub == 0) return LX3C_OK;
  L.sub_pair.resize(sub.size());
  for (size_t i = 0; i < sub.size(); ++i) L.sub_pair[i] = sub[i].x;
  const int l1 = orient ? p->lb : p->la, l2 = orient ? p->la : p->lb;
  const ClassTables* ct;
  try {
    ct = &class_tables(l1, l2, p->lc, p->bra_pure);
  } catch (std::exception& e) {
    return fail(LX3C_ENOTSUP, std::string("eri3c_plan: ") + e.what());
  }
  DevClass* dc;
  lx3c_status rc = device_class(ds, *ct, &dc);
  if (rc) return rc;
  ClassDesc& d = L.desc;
  if (fill_class_desc(d, *ct, *dc, ds, orient, kmax, p->Ka * p->Kb, p->Kc, p->naux) < 0)
    return fail(LX3C_ENOTSUP, "eri3c_plan: class does not fit in shared memory");
  d.npair = p->npair; d.naux = p->naux;
  d.ntile_aux = (int)((p->naux + d.T - 1) / d.T);
  d.nsub = L.nsub;
  d.ntiles = L.nsub * d.ntile_aux;
  int occ = eri3c_occupancy(d.smem_doubles * 8);
  L.grid = (int)std::min<long long>(d.ntiles, (long long)ds->nsm * occ * 8);
  CUDA_TRY(cudaMalloc(&L.d_sub, sub.size() * sizeof(int4)));
  CUDA_TRY(cudaMalloc(&L.d_prim, std::max<size_t>(prim.size(), 1) * sizeof(int)));
  CUDA_TRY(cudaMemcpyAsync(L.d_sub, sub.data(), sub.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
  if (!prim.empty())
    CUDA_TRY(cudaMemcpyAsync(L.d_prim, prim.data(), prim.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  d.subpairs = L.d_sub;
  d.primidx = L.d_prim;
  return LX3C_OK;
}

}  // namespace

lx3c_status lx3c_eri3c_plan(lx3c_plan** out, const lx3c_basis* orb, const lx3c_basis* aux, const int32_t* pairs,
                            int64_t npair, const int32_t* auxs, int64_t naux, int bra_pure, void* stream) {
  if (!out) return fail(LX3C_EINVAL, "eri3c_plan: null output pointer");
  *out = nullptr;
  if (!orb || !aux) return fail(LX3C_EINVAL, "eri3c_plan: null basis");
  if (npair <= 0 || naux <= 0) return fail(LX3C_EINVAL, "eri3c_plan: empty pair or aux list");
  if (!pairs || !auxs) return fail(LX3C_EINVAL, "eri3c_plan: null list");
  if (npair > (1LL << 31) - 1 || naux > (1LL << 31) - 1) return fail(LX3C_ENOTSUP, "eri3c_plan: list too long");
  int la = -1, lb = -1, lc = -1, Ka = 0, Kb = 0, Kc = 0;
  for (int64_t i = 0; i < npair; ++i) {
    int32_t a = pairs[2 * i], b = pairs[2 * i + 1];
    if (a < 0 || a >= orb->nshell || b < 0 || b >= orb->nshell)
      return fail(LX3C_EINVAL, "eri3c_plan: pair " + std::to_string(i) + " index out of range");
    if (i == 0) { la = orb->l[a]; lb = orb->l[b]; Ka = orb->k[a]; Kb = orb->k[b]; }
    if (orb->l[a] != la || orb->l[b] != lb || orb->k[a] != Ka || orb->k[b] != Kb)
      return fail(LX3C_EINVAL, "eri3c_plan: mixed (l, K) in pair list at " + std::to_string(i));
  }
  for (int64_t i = 0; i < naux; ++i) {
    int32_t c = auxs[i];
    if (c < 0 || c >= aux->nshell) return fail(LX3C_EINVAL, "eri3c_plan: aux index out of range");
    if (i == 0) { lc = aux->l[c]; Kc = aux->k[c]; }
    if (aux->l[c] != lc || aux->k[c] != Kc) return fail(LX3C_EINVAL, "eri3c_plan: mixed (l, K) in aux list");
  }
  if (la > LX3C_LMAX_ORB || lb > LX3C_LMAX_ORB || lc > LX3C_LMAX_AUX)
    return fail(LX3C_ENOTSUP, "eri3c_plan: angular momentum beyond the supported limits");
  DevState* ds;
  lx3c_status rc = device_state(&ds);
  if (rc) return rc;
  std::unique_ptr<lx3c_plan> p(new lx3c_plan);
  p->orb = orb;
  p->aux = aux;
  p->la = la; p->lb = lb; p->lc = lc; p->bra_pure = bra_pure ? 1 : 0;
  p->Ka = Ka; p->Kb = Kb; p->Kc = Kc;
  p->npair = npair; p->naux = naux;
  {
    const ClassTables& ct = class_tables(la, lb, lc, p->bra_pure);
    p->nblk = (int64_t)ct.nA * ct.nB * ct.nC;
  }
  std::vector<int4> subA, subB;
  std::vector<int> primA, primB;
  int kA = 0, kB = 0;
  for (int64_t i = 0; i < npair; ++i) {
    int oa = (int)primA.size(), ob = (int)primB.size();
    split_orientation(orb, pairs[2 * i], pairs[2 * i + 1], la, lb, primA, primB);
    int na = (int)primA.size() - oa, nb = (int)primB.size() - ob;
    if (na) subA.push_back(int4{(int)i, oa, na, 0});
    if (nb) subB.push_back(int4{(int)i, ob, nb, na > 0 ? 1 : 0});
    kA = std::max(kA, na);
    kB = std::max(kB, nb);
  }
  {
    // the flops the two launches execute: each sub-pair's primitive pairs
    // through its orientation's primitive stages, and once per sub-pair and
    // ket shell its contracted stages
    const ClassTables& ta = class_tables(la, lb, lc, p->bra_pure);
    const ClassTables& tb = class_tables(lb, la, lc, p->bra_pure);
    double f = 0;
    for (auto& s4 : subA) f += ta.flops_prim * s4.z * Kc + ta.flops_contr;
    for (auto& s4 : subB) f += tb.flops_prim * s4.z * Kc + tb.flops_contr;
    p->flops = f * (double)naux;
  }
  cudaStream_t st = (cudaStream_t)stream;
  rc = make_launch(ds, p.get(), 0, subA, primA, kA, st);
  if (!rc) rc = make_launch(ds, p.get(), 1, subB, primB, kB, st);
  if (rc) return rc;
  const int Kab = Ka * Kb;
  CUDA_TRY(cudaMalloc(&p->d_pairs, npair * 8));
  CUDA_TRY(cudaMalloc(&p->d_auxs, naux * 4));
  CUDA_TRY(cudaMalloc(&p->d_pairrec, (size_t)npair * Kab * kPairRec * 8));
  CUDA_TRY(cudaMalloc(&p->d_pairab, (size_t)npair * 3 * 8));
  CUDA_TRY(cudaMalloc(&p->d_auxrec, (size_t)naux * Kc * kAuxRec * 8));
  CUDA_TRY(cudaMalloc(&p->d_auxc, (size_t)naux * 3 * 8));
  CUDA_TRY(cudaMemcpyAsync(p->d_pairs, pairs, npair * 8, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(p->d_auxs, auxs, naux * 4, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (auto& L : p->L) {
    L.desc.pairrec = p->d_pairrec; L.desc.pairab = p->d_pairab;
    L.desc.auxrec = p->d_auxrec; L.desc.auxc = p->d_auxc;
  }
  *out = p.release();
  return LX3C_OK;
}

lx3c_status lx3c_eri3c_execute(lx3c_plan* p, double* out, void* stream) {
  if (!p) return fail(LX3C_EINVAL, "eri3c_execute: null plan");
  if (!out) return fail(LX3C_EINVAL, "eri3c_execute: null output");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(launch_pair_precompute(p->orb->dev(), p->d_pairs, p->npair, p->Ka, p->Kb, p->d_pairrec, p->d_pairab, st));
  CUDA_TRY(launch_aux_precompute(p->aux->dev(), p->d_auxs, p->naux, p->Kc, p->d_auxrec, p->d_auxc, st));
  for (auto& L : p->L) {
    if (!L.nsub) continue;
    ClassDesc d = L.desc;
    d.out = out;
    CUDA_TRY(launch_eri3c(d, L.grid, st));
  }
  return LX3C_OK;
}

lx3c_status lx3c_plan_info(const lx3c_plan* p, int64_t* out, int n) {
  if (!p || (!out && n > 0)) return fail(LX3C_EINVAL, "plan_info: null pointer");
  std::vector<int64_t> v;
  v.push_back(2 + (p->L[0].nsub > 0) + (p->L[1].nsub > 0));
  for (auto& l : p->L) {
    v.push_back(l.nsub);
    v.push_back(l.desc.T);
    v.push_back(l.desc.G);
    v.push_back(l.desc.mode);
    v.push_back((int64_t)l.desc.smem_doubles * 8);
    v.push_back(l.grid);
  }
  v.push_back((int64_t)std::llround(p->flops));
  for (int i = 0; i < n && i < (int)v.size(); ++i) out[i] = v[i];
  return LX3C_OK;
}

lx3c_status lx3c_plan_sizes(const lx3c_plan* p, int64_t* block, int64_t* total) {
  if (!p) return fail(LX3C_EINVAL, "plan_sizes: null plan");
  if (block) *block = p->nblk;
  if (total) *total = (int64_t)p->npair * p->naux * p->nblk;
  return LX3C_OK;
}

lx3c_status lx3c_eri3c_host(int64_t orb_nshell, const int32_t* orb_l, const int32_t* orb_k, const double* orb_xyz,
                            const double* orb_exps, const double* orb_coefs, int64_t aux_nshell,
                            const int32_t* aux_l, const int32_t* aux_k, const double* aux_xyz,
                            const double* aux_exps, const double* aux_coefs, const int32_t* pairs, int64_t npair,
                            const int32_t* auxs, int64_t naux, int bra_pure, double* out_host, void* stream) {
  if (!out_host) return fail(LX3C_EINVAL, "eri3c_host: null output");
  lx3c_basis *orb = nullptr, *aux = nullptr;
  lx3c_plan* plan = nullptr;
  double* d_out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  lx3c_status rc = lx3c_basis_create(&orb, orb_nshell, orb_l, orb_k, orb_xyz, nullptr, orb_exps, orb_coefs, stream);
  if (!rc) rc = lx3c_basis_create(&aux, aux_nshell, aux_l, aux_k, aux_xyz, nullptr, aux_exps, aux_coefs, stream);
  if (!rc) rc = lx3c_eri3c_plan(&plan, orb, aux, pairs, npair, auxs, naux, bra_pure, stream);
  int64_t total = 0;
  if (!rc) rc = lx3c_plan_sizes(plan, nullptr, &total);
  // Pair-range chunks of about 512 MB alternate between two device buffers;
  // each finished chunk is copied to the host on a second stream while the
  // next one is computed.  Buffers, stream and events persist per device.
  DevState* ds = nullptr;
  if (!rc) rc = device_state(&ds);
  std::unique_lock<std::mutex> hl;
  if (ds) hl = std::unique_lock<std::mutex>(ds->host_mu);
  cudaStream_t cs = nullptr;
  cudaEvent_t* done = ds ? ds->host_done : nullptr;
  cudaEvent_t* freed = ds ? ds->host_freed : nullptr;
  const long long per_pair = plan ? plan->naux * plan->nblk : 0;
  long long cp = 1;
  if (!rc && total > 0) {
    cp = std::max(1LL, std::min<long long>(npair, (512LL << 20) / 8 / std::max(1LL, per_pair)));
    const size_t need = (size_t)(2 * cp * per_pair);
    cudaError_t e = cudaSuccess;
    if (ds->host_cap < need) {
      cudaFree(ds->host_buf);
      ds->host_buf = nullptr;
      ds->host_cap = 0;
      e = cudaMalloc(&ds->host_buf, need * 8);
      if (e == cudaSuccess) ds->host_cap = need;
    }
    if (e != cudaSuccess) rc = fail(LX3C_ENOMEM, "eri3c_host: device output allocation failed");
    d_out = ds->host_buf;
  }
  if (!rc && total > 0) {
    cudaError_t e = cudaSuccess;
    if (!ds->host_cs) e = cudaStreamCreateWithFlags(&ds->host_cs, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      if (!done[b]) e = cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming);
      if (e == cudaSuccess && !freed[b]) e = cudaEventCreateWithFlags(&freed[b], cudaEventDisableTiming);
    }
    cs = ds->host_cs;
    if (e == cudaSuccess) e = launch_pair_precompute(plan->orb->dev(), plan->d_pairs, plan->npair, plan->Ka, plan->Kb,
                                                     plan->d_pairrec, plan->d_pairab, st);
    if (e == cudaSuccess) e = launch_aux_precompute(plan->aux->dev(), plan->d_auxs, plan->naux, plan->Kc, plan->d_auxrec,
                                                    plan->d_auxc, st);
    int c = 0;
    for (long long p0 = 0; p0 < npair && e == cudaSuccess; p0 += cp, ++c) {
      const long long p1 = std::min<long long>(npair, p0 + cp);
      const int b = c & 1;
      double* buf = d_out + (size_t)b * cp * per_pair;
      if (c >= 2) e = cudaStreamWaitEvent(st, freed[b], 0);
      for (auto& L : plan->L) {
        if (!L.nsub || e != cudaSuccess) continue;
        const long long s0 = std::lower_bound(L.sub_pair.begin(), L.sub_pair.end(), (int)p0) - L.sub_pair.begin();
        const long long s1 = std::lower_bound(L.sub_pair.begin(), L.sub_pair.end(), (int)p1) - L.sub_pair.begin();
        if (s1 <= s0) continue;
        ClassDesc d = L.desc;
        d.out = buf;
        d.out_pair0 = p0;
        d.subpairs = L.d_sub + s0;
        d.nsub = s1 - s0;
        d.ntiles = d.nsub * d.ntile_aux;
        e = launch_eri3c(d, (int)std::min<long long>(L.grid, d.ntiles), st);
      }
      if (e == cudaSuccess) e = cudaEventRecord(done[b], st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, done[b], 0);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_host + p0 * per_pair, buf, (size_t)((p1 - p0) * per_pair) * 8, cudaMemcpyDeviceToHost, cs);
      if (e == cudaSuccess) e = cudaEventRecord(freed[b], cs);
    }
    cudaError_t e2 = cudaStreamSynchronize(cs);
    if (e == cudaSuccess) e = e2;
    e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) rc = fail(LX3C_ECUDA, std::string("eri3c_host: ") + cudaGetErrorString(e));
  }

  lx3c_plan_destroy(plan);
  lx3c_basis_destroy(orb);
  lx3c_basis_destroy(aux);
  return rc;
}

lx3c_status lx3c_boys(const double* T, int64_t n, int mmax, double* out, void* stream) {
  if (n < 0 || mmax < 0 || mmax > kBoysMmax) return fail(LX3C_EINVAL, "boys: bad n or mmax");
  if (n > 0 && (!T || !out)) return fail(LX3C_EINVAL, "boys: null pointer");
  DevState* ds;
  lx3c_status rc = device_state(&ds);
  if (rc) return rc;
  CUDA_TRY(launch_boys(T, n, mmax, ds->boys_tab, ds->boys_mid, boys_large_const(mmax), out, (cudaStream_t)stream));
  return LX3C_OK;
}

lx3c_status lx3c_class_tables_check(int la, int lb, int lc, int bra_pure) {
  if (la < 0 || lb < 0 || lc < 0 || la > LX3C_LMAX_ORB + 1 || lb > LX3C_LMAX_ORB + 1 || lc > LX3C_LMAX_AUX)
    return fail(LX3C_EINVAL, "class_tables_check: bad argument");
  try {
    const std::string msg = check_class_tables(class_tables(la, lb, lc, bra_pure ? 1 : 0));
    if (!msg.empty()) return fail(LX3C_EINVAL, "class tables: " + msg);
  } catch (std::exception& e) {
    return fail(LX3C_ENOTSUP, e.what());
  }
  return LX3C_OK;
}

lx3c_status lx3c_set_orientation_threshold(double amp_max) {
  if (!(amp_max == 0.0 || (amp_max >= 1.0 && std::isfinite(amp_max))))
    return fail(LX3C_EINVAL, "set_orientation_threshold: amp_max must be 0 (default) or a finite value >= 1");
  g_amp_max.store(amp_max == 0.0 ? kDefaultAmpMax : amp_max);
  return LX3C_OK;
}

lx3c_status lx3c_set_compensation(int bits) {
  if (bits < 0 || bits > 3) return fail(LX3C_EINVAL, "set_compensation: bits must be in 0..3");
  g_comp_bits.store(bits);
  return LX3C_OK;
}

lx3c_status lx3c_hrr_tables_check(int la, int lb, int lc, int bra_pure, int variant, const double* AB,
                                  double* max_rel_err) {
  if (!AB || !max_rel_err || la < 0 || lb < 0 || lc < 0 || la > LX3C_LMAX_ORB + 1 || lb > LX3C_LMAX_ORB + 1 ||
      lc > LX3C_LMAX_AUX || variant < 0 || variant > 1)
    return fail(LX3C_EINVAL, "hrr_tables_check: bad argument");
  try {
    const ClassTables& ct = class_tables_variant(la, lb, lc, bra_pure ? 1 : 0, variant);
    const std::string msg = check_class_tables(ct);
    if (!msg.empty()) return fail(LX3C_EINVAL, "class tables: " + msg);
    *max_rel_err = hrr_moment_error(ct, AB);
  } catch (std::exception& e) {
    return fail(LX3C_ENOTSUP, e.what());
  }
  return LX3C_OK;
}

lx3c_status lx3c_hrr_hint(int la, int lb, int lc, int bra_pure, int variant) {
  if (la < 0 || lb < 0 || lc < 0 || la > LX3C_LMAX_ORB + 1 || lb > LX3C_LMAX_ORB + 1 || lc > LX3C_LMAX_AUX ||
      variant < -1 || variant > 1)
    return fail(LX3C_EINVAL, "hrr_hint: bad argument");
  set_hrr_hint(la, lb, lc, bra_pure, variant);
  return LX3C_OK;
}

lx3c_status lx3c_shape_hint(int la, int lb, int lc, int bra_pure, int kab, int kc, int ctas_per_sm) {
  if (la < 0 || lb < 0 || lc < 0 || la > LX3C_LMAX_ORB + 1 || lb > LX3C_LMAX_ORB + 1 || lc > LX3C_LMAX_AUX ||
      kab < 1 || kc < 1 || ctas_per_sm < 0 || ctas_per_sm > 3)
    return fail(LX3C_EINVAL, "shape_hint: bad argument");
  set_shape_hint(la, lb, lc, bra_pure, kab, kc, ctas_per_sm);
  return LX3C_OK;
}

lx3c_status lx3c_tile_hint(int la, int lb, int lc, int bra_pure, int kab, int kc, int T, int G) {
  if (la < 0 || lb < 0 || lc < 0 || la > LX3C_LMAX_ORB + 1 || lb > LX3C_LMAX_ORB + 1 || lc > LX3C_LMAX_AUX ||
      kab < 1 || kc < 1 || T < 0 || T > 512 || (T > 0 && (G < 1 || G > kab * kc)))
    return fail(LX3C_EINVAL, "tile_hint: bad argument");
  set_tile_hint(la, lb, lc, bra_pure, kab, kc, T, G);
  return LX3C_OK;
}

lx3c_status lx3c_shape_query(int la, int lb, int lc, int bra_pure, int kab, int kc, int64_t naux, int ctas_per_sm,
                             int32_t* out) {
  if (!out || la < 0 || lb < 0 || lc < 0 || la > LX3C_LMAX_ORB + 1 || lb > LX3C_LMAX_ORB + 1 ||
      lc > LX3C_LMAX_AUX || kab < 1 || kc < 1 || naux < 1 || ctas_per_sm < 0 || ctas_per_sm > 3)
    return fail(LX3C_EINVAL, "shape_query: bad argument");
  try {
    const ClassTables& ct = class_tables(la, lb, lc, bra_pure ? 1 : 0);
    const int smem = 233472;  // shared memory per SM of the target (GB300)
    LaunchShape sh = ctas_per_sm ? choose_shape_for(ct, kab, kc, naux, smem, ctas_per_sm)
                                 : choose_shape(ct, kab, kc, naux, smem);
    out[0] = sh.T; out[1] = sh.G; out[2] = sh.mode; out[3] = sh.smem_bytes;
  } catch (std::exception& e) {
    return fail(LX3C_ENOTSUP, e.what());
  }
  return LX3C_OK;
}

lx3c_status lx3c_class_flops(int la, int lb, int lc, int Kab, int Kc, int bra_pure, double* flops) {
  if (!flops || la < 0 || lb < 0 || lc < 0 || la > LX3C_LMAX_ORB || lb > LX3C_LMAX_ORB || lc > LX3C_LMAX_AUX ||
      Kab < 1 || Kc < 1)
    return fail(LX3C_EINVAL, "class_flops: bad argument");
  try {
    const ClassTables& ct = class_tables(la, lb, lc, bra_pure ? 1 : 0);
    *flops = ct.flops_prim * (double)Kab * Kc + ct.flops_contr;
  } catch (std::exception& e) {
    return fail(LX3C_ENOTSUP, e.what());
  }
  return LX3C_OK;
}

lx3c_status lx3c_solid_harmonics(int l, double* out) {
  if (l < 0 || l > 12 || !out) return fail(LX3C_EINVAL, "solid_harmonics: bad argument");
  auto T = solid_matrix(l);
  std::memcpy(out, T.data(), T.size() * 8);
  return LX3C_OK;
}

lx3c_status lx3c_cvrr2_expansion(const int32_t* a, const int32_t* c, int32_t cap, double* terms, int32_t* nterms) {
  if (!a || !c || !nterms || (cap > 0 && !terms)) return fail(LX3C_EINVAL, "cvrr2_expansion: null pointer");
  for (int i = 0; i < 3; ++i)
    if (a[i] < 0 || c[i] < 0) return fail(LX3C_EINVAL, "cvrr2_expansion: negative exponent");
  int la = a[0] + a[1] + a[2], lc = c[0] + c[1] + c[2];
  if (la > 2 * LX3C_LMAX_ORB || lc > LX3C_LMAX_AUX) return fail(LX3C_ENOTSUP, "cvrr2_expansion: too large");
  // the class (la, 0 | lc) contains the target (a 0|c) at level 0
  const ClassTables* ct;
  try {
    ct = &class_tables(la, 0, lc, 0);
  } catch (std::exception& e) {
    return fail(LX3C_ENOTSUP, e.what());
  }
  int row = cart_index(a[0], a[1], a[2]);
  int id = row * ct->ncc + cart_index(c[0], c[1], c[2]);
  int q0 = ct->gptr[id], q1 = ct->gptr[id + 1];
  *nterms = q1 - q0;
  for (int q = q0; q < q1 && q - q0 < cap; ++q) {
    unsigned e = ct->gterm[q];
    const int4 key = ct->acc_key[e & 0xFFFFF];
    int el = key.x >> 16, ei = key.x & 0xFFFF, nl = key.z >> 16, ni = key.z & 0xFFFF;
    // decode component indices back to exponents
    auto decode = [](int l, int idx, double* o) {
      int i = 0;
      for (int x = l; x >= 0; --x)
        for (int y = l - x; y >= 0; --y) {
          if (i == idx) { o[0] = x; o[1] = y; o[2] = l - x - y; return; }
          ++i;
        }
    };
    double* t = terms + 8 * (q - q0);
    decode(el, ei, t);
    t[3] = key.y;
    decode(nl, ni, t + 4);
    t[7] = ct->pal[e >> 20];
  }
  return LX3C_OK;
}

}  // extern "C"
