// lx3c_eri3c_noalloc: the (ab|C) class evaluation without any device memory
// allocation, for callers that cannot call cudaMalloc/cudaFree around the call
// (see include/lx3c.h).  Every device buffer the path needs beyond the
// caller's inputs and output (primitive-pair and ket-primitive records, the
// oriented sub-pair lists, the Boys table and the class index tables) lives in
// one file-scope __device__ array, and the existing precompute and integral
// kernels are launched on it unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
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
int eri3c_occupancy(int smem_bytes);
void set_last_error(const std::string& msg);
}  // namespace lx3c

using namespace lx3c;

namespace {

// Limits of the shared scratch array (all counts inclusive).
constexpr long long kMaxPrimPairs = 1LL << 16;  // npair * ka * kb
constexpr long long kMaxPairs = 1LL << 16;      // npair
constexpr long long kMaxAuxPrims = 1LL << 16;   // naux * kc (and naux)
constexpr size_t kTableBytes = 4u << 20;        // class index tables

// Byte layout of the scratch array (offsets are multiples of 256).
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffPairRec = 0;
constexpr size_t kOffPairAB = align256(kOffPairRec + sizeof(double) * kMaxPrimPairs * kPairRec);
constexpr size_t kOffAuxRec = align256(kOffPairAB + sizeof(double) * kMaxPairs * 3);
constexpr size_t kOffAuxC = align256(kOffAuxRec + sizeof(double) * kMaxAuxPrims * kAuxRec);
constexpr size_t kOffSub = align256(kOffAuxC + sizeof(double) * kMaxAuxPrims * 3);
constexpr size_t kOffPrim = align256(kOffSub + sizeof(int4) * 2 * kMaxPairs);
constexpr size_t kOffBoys = align256(kOffPrim + sizeof(int) * 2 * kMaxPrimPairs);
constexpr size_t kOffBoysMid = align256(kOffBoys + sizeof(double) * kBoysNInt * kBoysNF * 8);
constexpr size_t kOffTables = align256(kOffBoysMid + sizeof(double) * kBoysNInt);
constexpr size_t kScratchBytes = align256(kOffTables + kTableBytes);  // about 27 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

lx3c_status na_fail(lx3c_status s, const std::string& m) {
  set_last_error("eri3c_noalloc: " + m);
  return s;
}

std::mutex g_na_mu;
std::map<int, unsigned char*> g_na_base;  // per device: scratch address, set up once
std::vector<double> g_na_boys, g_na_mid;

// Split the primitive pairs of every pair by orientation with the planned
// path's rule (split_orientation): a pair keeps one orientation, the one with
// the smaller worst weighted HRR amplification, when that is at most amp_max;
// otherwise each primitive pair runs on its more compact centre.  Sub-pair p of list o holds
// its primitive indices at prim[o][p*kab ...].  A sub-pair with no primitive
// pairs is skipped by the integral kernel; list 1 accumulates onto list 0's
// store only where list 0 has primitive pairs for that pair.
__global__ void noalloc_orient(const int32_t* __restrict__ pairs, long long npair, int la, int lb, int ka, int kb,
                               const int64_t* __restrict__ off, const double* __restrict__ xyz,
                               const double* __restrict__ exps, const double* __restrict__ coefs, double amp_max,
                               int4* __restrict__ sub, int* __restrict__ prim) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= npair) return;
  const int kab = ka * kb;
  const int sa = pairs[2 * p], sb = pairs[2 * p + 1];
  double ab2 = 0;
  for (int x = 0; x < 3; ++x) ab2 += (xyz[3 * sa + x] - xyz[3 * sb + x]) * (xyz[3 * sa + x] - xyz[3 * sb + x]);
  const double dab = sqrt(ab2);
  double wmax = 0;
  for (int ia = 0; ia < ka; ++ia)
    for (int ib = 0; ib < kb; ++ib) {
      const double za = exps[off[sa] + ia], zb = exps[off[sb] + ib], g = za + zb;
      wmax = fmax(wmax, fabs(coefs[off[sa] + ia] * coefs[off[sb] + ib]) * exp(-za * zb / g * ab2) / g);
    }
  double worstA = 0, worstB = 0;
  for (int ia = 0; ia < ka; ++ia)
    for (int ib = 0; ib < kb; ++ib) {
      const double za = exps[off[sa] + ia], zb = exps[off[sb] + ib], g = za + zb;
      const double w = fabs(coefs[off[sa] + ia] * coefs[off[sb] + ib]) * exp(-za * zb / g * ab2) / g;
      const double f = wmax > 0 ? w / wmax : 1.0, sg = 1.0 / sqrt(2.0 * g);
      worstA = fmax(worstA, pow((dab + sg) / (za / g * dab + sg), (double)lb) * f);
      worstB = fmax(worstB, pow((dab + sg) / (zb / g * dab + sg), (double)la) * f);
    }
  int whole = -1;
  if (lb == 0) whole = 0;
  else if (fmin(worstA, worstB) <= amp_max) whole = worstB < worstA ? 1 : 0;
  int na = 0, nb = 0;
  for (int ia = 0; ia < ka; ++ia)
    for (int ib = 0; ib < kb; ++ib) {
      const bool onB = whole >= 0 ? whole == 1 : exps[off[sb] + ib] > exps[off[sa] + ia];
      if (onB) prim[(npair + p) * kab + nb++] = ia * kb + ib;
      else prim[p * kab + na++] = ia * kb + ib;
    }
  sub[p] = int4{(int)p, (int)(p * kab), na, 0};
  sub[npair + p] = int4{(int)p, (int)(p * kab), nb, na > 0 ? 1 : 0};
}

// Host copy of both orientations' class tables, one blob per class, made on
// first use and kept until process exit.
struct NaBlob {
  std::vector<char> bytes;
  size_t base[2] = {0, 0};
  size_t offs[2][18] = {};
};

const NaBlob& na_blob(int la, int lb, int lc, int bra_pure, int split) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int, int>, NaBlob> cache;
  std::lock_guard<std::mutex> lk(mu);
  const ClassTables* ct[2] = {&class_tables(la, lb, lc, bra_pure), &class_tables(lb, la, lc, bra_pure)};
  auto key = std::make_tuple(la, lb, lc, bra_pure, ct[0]->hrr2, ct[1]->hrr2);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  NaBlob nb;
  for (int o = 0; o < 1 + split; ++o) {
    std::vector<char> part = class_blob(*ct[o], nb.offs[o]);
    nb.base[o] = (nb.bytes.size() + 255) & ~size_t(255);
    nb.bytes.resize(nb.base[o] + part.size());
    std::memcpy(nb.bytes.data() + nb.base[o], part.data(), part.size());
  }
  return cache.emplace(key, std::move(nb)).first->second;
}

}  // namespace

extern "C" lx3c_status lx3c_eri3c_noalloc(int la, int lb, int lc, int ka, int kb, int kc, int bra_pure,
                                          const int64_t* orb_off, const double* orb_xyz, const double* orb_exps,
                                          const double* orb_coefs, const int64_t* aux_off, const double* aux_xyz,
                                          const double* aux_exps, const double* aux_coefs, const int32_t* pairs,
                                          int64_t npair, const int32_t* auxs, int64_t naux, double* out,
                                          void* stream) {
  if (la < 0 || lb < 0 || lc < 0 || la > LX3C_LMAX_ORB || lb > LX3C_LMAX_ORB || lc > LX3C_LMAX_AUX)
    return na_fail(LX3C_ENOTSUP, "angular momentum beyond the supported limits");
  if (ka < 1 || kb < 1 || kc < 1 || ka > LX3C_KMAX || kb > LX3C_KMAX || kc > LX3C_KMAX)
    return na_fail(LX3C_ENOTSUP, "contraction degree beyond the supported limits");
  if (npair <= 0 || naux <= 0) return na_fail(LX3C_EINVAL, "empty pair or ket list");
  if (!orb_off || !orb_xyz || !orb_exps || !orb_coefs || !aux_off || !aux_xyz || !aux_exps || !aux_coefs ||
      !pairs || !auxs || !out)
    return na_fail(LX3C_EINVAL, "null pointer");
  if (npair > kMaxPairs || npair * ka * kb > kMaxPrimPairs || naux > kMaxAuxPrims || naux * kc > kMaxAuxPrims)
    return na_fail(LX3C_ENOTSUP, "problem exceeds the scratch limits (npair <= 65536, npair*ka*kb <= 65536, "
                                 "naux*kc <= 65536)");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(LX3C_ECUDA, cudaGetErrorString(e));
  unsigned char* base = nullptr;
  {
    // Set-up, once per device with that device current: the host only holds a
    // stand-in symbol for the array, so its device address is looked up here;
    // the Boys table is copied into it once.
    std::lock_guard<std::mutex> lk(g_na_mu);
    auto it = g_na_base.find(dev);
    if (it == g_na_base.end()) {
      e = cudaGetSymbolAddress((void**)&base, g_noalloc_scratch);
      if (e != cudaSuccess)
        return na_fail(LX3C_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      if (g_na_boys.empty()) boys_tables(g_na_boys, g_na_mid);
      e = cudaMemcpy(base + kOffBoys, g_na_boys.data(), g_na_boys.size() * 8, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(base + kOffBoysMid, g_na_mid.data(), g_na_mid.size() * 8,
                                           cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = init_constants();
      if (e != cudaSuccess) return na_fail(LX3C_ECUDA, cudaGetErrorString(e));
      g_na_base[dev] = base;
    } else {
      base = it->second;
    }
  }
  int nsm = 0, smem = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const int kab = ka * kb;
  const int split = lb > 0 ? 1 : 0;
  double* pairrec = (double*)(base + kOffPairRec);
  double* pairab = (double*)(base + kOffPairAB);
  double* auxrec = (double*)(base + kOffAuxRec);
  double* auxc = (double*)(base + kOffAuxC);
  int4* sub = (int4*)(base + kOffSub);
  int* prim = (int*)(base + kOffPrim);
  // class tables of both orientations, packed into the table region from a
  // host copy kept for the life of the process (the copy's source outlives
  // the call).  The source is pageable memory: CUDA stages the copy, so this
  // call may wait for work already queued on st before it returns.
  const ClassTables* cts[2];
  const NaBlob* nb = nullptr;
  try {
    cts[0] = &class_tables(la, lb, lc, bra_pure ? 1 : 0);
    cts[1] = &class_tables(lb, la, lc, bra_pure ? 1 : 0);
    nb = &na_blob(la, lb, lc, bra_pure ? 1 : 0, split);
  } catch (std::exception& ex) {
    return na_fail(LX3C_ENOTSUP, ex.what());
  }
  if (nb->bytes.size() > kTableBytes) return na_fail(LX3C_ENOTSUP, "class tables exceed the scratch table region");
  unsigned char* tb = base + kOffTables;
  e = cudaMemcpyAsync(tb, nb->bytes.data(), nb->bytes.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return na_fail(LX3C_ECUDA, cudaGetErrorString(e));
  DevBasis orb{nullptr, nullptr, orb_off, orb_xyz, orb_exps, orb_coefs};
  DevBasis aux{nullptr, nullptr, aux_off, aux_xyz, aux_exps, aux_coefs};
  e = launch_pair_precompute(orb, pairs, npair, ka, kb, pairrec, pairab, st);
  if (e == cudaSuccess) e = launch_aux_precompute(aux, auxs, naux, kc, auxrec, auxc, st);
  if (e == cudaSuccess) {
    noalloc_orient<<<(unsigned)((npair + 127) / 128), 128, 0, st>>>(pairs, npair, la, lb, ka, kb, orb_off, orb_xyz,
                                                                     orb_exps, orb_coefs, orientation_amp_max(), sub, prim);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return na_fail(LX3C_ECUDA, cudaGetErrorString(e));
  for (int o = 0; o < 1 + split; ++o) {
    const ClassTables& ct = *cts[o];
    LaunchShape sh = choose_shape(ct, kab, kc, naux, smem);
    if (sh.smem_bytes < 0 || sh.smem_bytes > 232448) return na_fail(LX3C_ENOTSUP, "class does not fit in shared memory");
    DevClass dc;
    class_blob_pointers(dc, tb + nb->base[o], nb->offs[o]);
    ClassDesc d;
    fill_desc_common(d, ct, dc, (const double*)(base + kOffBoys), (const double*)(base + kOffBoysMid), o, kab, kab,
                     kc, sh);
    d.npair = npair; d.naux = naux;
    d.ntile_aux = (int)((naux + d.T - 1) / d.T);
    d.nsub = npair;
    d.ntiles = npair * d.ntile_aux;
    d.subpairs = sub + o * npair;
    d.primidx = prim + (size_t)o * npair * kab;
    d.pairrec = pairrec; d.pairab = pairab; d.auxrec = auxrec; d.auxc = auxc;
    d.out = out;
    const int occ = eri3c_occupancy(d.smem_doubles * 8);
    const int grid = (int)std::min<long long>(d.ntiles, (long long)nsm * occ * 8);
    e = launch_eri3c(d, grid, st);
    if (e != cudaSuccess) return na_fail(LX3C_ECUDA, cudaGetErrorString(e));
  }
  return LX3C_OK;
}
