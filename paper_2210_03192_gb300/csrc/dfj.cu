// Density-fitted Coulomb build (paper Sec. 3: a DF-J builder fed by an
// integral-digestion callable, so that integrals never reach global memory):
//   gamma_P = sum_{mu nu} (mu nu|P) D_{mu nu},   J_{mu nu} = sum_P (mu nu|P) c_P
// over all AO pairs (mu, nu) of a solid-harmonic orbital basis, evaluated on
// unique shell pairs a <= b (off-diagonal pairs weighted twice in gamma and
// mirrored into J).
//
// Setup (lx3c_dfj_plan): Schwarz-type screening estimates Q_ab, Q_P; every
// (la lb | lc) class group keeps its ket shells sorted by Q_P so that the
// ket shells surviving Q_ab Q_P >= tol for a pair form a prefix of the list;
// tiles (sub-pair, ket range) are tabulated.  Execution runs the class kernel
// in digest mode: gamma and J are accumulated from each tile's block in
// shared memory into exact fixed-point accumulators (fixed128.cuh), so the
// result does not depend on the order of the contributions; final kernels
// convert them to FP64 and symmetrise J.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lx3c.h"
#include "fixed128.cuh"
#include "lx3c_internal.h"

namespace lx3c {
cudaError_t launch_pair_precompute(const DevBasis& orb, const int32_t* pairs, long long npair, int Ka, int Kb,
                                   double* rec, double* ab, cudaStream_t st, int scale_a = 0, int scale_b = 0);
cudaError_t launch_aux_precompute(const DevBasis& aux, const int32_t* auxs, long long naux, int Kc, double* rec,
                                  double* cxyz, cudaStream_t st);
cudaError_t launch_eri3c(const ClassDesc& d, int grid, cudaStream_t st);
int eri3c_occupancy(int smem_bytes);
cudaError_t launch_persistent(const ClassDesc* descs, const int2* work, long long nwork, unsigned long long* counter,
                              int grid, int smem_bytes, int three, cudaStream_t st);
cudaError_t launch_jeng_matrix(const ClassDesc& d, int grid, cudaStream_t st);
cudaError_t launch_jeng_pair(const ClassDesc& d, int finish, cudaStream_t st);
int persistent_occupancy(int smem_bytes, int three);
}  // namespace lx3c

using namespace lx3c;

namespace {

// Ket-count bound for the shape chooser from the tile fill: the largest T
// (a power of two up to 512) at which this launch's tiles hold at least 80%
// screened triples, returned as T/2 (the chooser allows T up to twice the
// count it is given), and never above the longest ket list.
long long fill_bound(const std::vector<int4>& sub, const std::vector<int>& counts, int cmax) {
  long long tot = 0;
  for (auto& s : sub) tot += counts[s.x];
  int pick = 1;
  for (int T = 512; T >= 1; T /= 2) {
    long long slots = 0;
    for (auto& s : sub) slots += (long long)((counts[s.x] + T - 1) / T) * T;
    if (tot * 5 >= slots * 4) { pick = T; break; }
  }
  return std::min<long long>(cmax, std::max(1, pick / 2));
}


lx3c_status dfail(lx3c_status s, const std::string& m) {
  set_last_error("dfj: " + m);
  return s;
}

#define DCUDA(expr)                                                                                      \
  do {                                                                                                   \
    cudaError_t e_ = (expr);                                                                             \
    if (e_ != cudaSuccess) return dfail(LX3C_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// J <- J + J^T (the digest accumulates each unique shell pair into one block;
// diagonal shell blocks carry half weight, so the sum is exact there too).
__global__ void symmetrize(double* J, long long n) {
  long long i = blockIdx.y * (long long)blockDim.y + threadIdx.y;
  long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n || j >= n || j < i) return;
  if (i == j) {
    J[i * n + i] *= 2.0;
  } else {
    const double s = J[i * n + j] + J[j * n + i];
    J[i * n + j] = s;
    J[j * n + i] = s;
  }
}

// out[i] = value of the fixed-point accumulator acc[i] (gamma, gradient)
__global__ void fix_finish(const unsigned long long* __restrict__ acc, long long n, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = fix_decode(acc + kFixWords * i);
}

// J[i][j] = A[i][j] + A[j][i] from the accumulated unique-pair blocks A (the
// digest adds each unique shell pair's block once, diagonal shell blocks
// with half weight, so this is exact on the diagonal too)
__global__ void fix_finish_J(const unsigned long long* __restrict__ acc, long long n, double* __restrict__ J) {
  const long long i = blockIdx.y * (long long)blockDim.y + threadIdx.y;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n && j < n) J[i * n + j] = fix_decode(acc + kFixWords * (i * n + j)) + fix_decode(acc + kFixWords * (j * n + i));
}

cudaError_t launch_fix_finish(const unsigned long long* acc, long long n, double* out, cudaStream_t st) {
  fix_finish<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(acc, n, out);
  return cudaGetLastError();
}

cudaError_t launch_fix_finish_J(const unsigned long long* acc, long long n, double* J, cudaStream_t st) {
  dim3 blk(32, 8), grd((unsigned)((n + 31) / 32), (unsigned)((n + 7) / 8));
  fix_finish_J<<<grd, blk, 0, st>>>(acc, n, J);
  return cudaGetLastError();
}

// energy = sum_i c_i gamma_i (one block, fixed-order tree reduction)
__global__ void dot_energy(const double* __restrict__ c, const double* __restrict__ g, long long n, double* out) {
  __shared__ double part[256];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += 256) s = fma(c[i], g[i], s);
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0];
}

constexpr double kPi = 3.14159265358979323846;

// sqrt of a Schwarz-type estimate of max |(ab|ab)| for a shell pair: the
// (ss|ss) value of each primitive pair times the rms size of (x-A)^la (x-B)^lb
// under the product Gaussian.
double q_pair_raw(int la, int ka, const double* A, const double* ea, const double* ca, int lb, int kb,
                  const double* B, const double* eb, const double* cb) {
  double ab2 = 0;
  for (int x = 0; x < 3; ++x) ab2 += (A[x] - B[x]) * (A[x] - B[x]);
  double q = 0;
  for (int ia = 0; ia < ka; ++ia)
    for (int ib = 0; ib < kb; ++ib) {
      const double za = ea[ia], zb = eb[ib], g = za + zb;
      double pa2 = 0, pb2 = 0;
      for (int x = 0; x < 3; ++x) {
        const double P = (za * A[x] + zb * B[x]) / g;
        pa2 += (P - A[x]) * (P - A[x]);
        pb2 += (P - B[x]) * (P - B[x]);
      }
      q += std::fabs(ca[ia] * cb[ib]) * std::exp(-za * zb / g * ab2) *
           std::sqrt(2.0 * std::pow(kPi, 2.5) / (g * g * std::sqrt(2.0 * g))) * std::pow(pa2 + 0.5 / g, 0.5 * la) *
           std::pow(pb2 + 0.5 / g, 0.5 * lb);
    }
  return q;
}

double q_aux_raw(int l, int k, const double* e, const double* c) {
  double q = 0;
  for (int i = 0; i < k; ++i)
    q += std::fabs(c[i]) * std::sqrt(2.0 * std::pow(kPi, 2.5) / (e[i] * e[i] * std::sqrt(2.0 * e[i]))) *
         std::pow(0.5 / e[i], 0.5 * l);
  return q;
}

double q_pair(const lx3c_basis* b, int sa, int sb) {
  return q_pair_raw(b->l[sa], b->k[sa], &b->xyz[3 * sa], &b->exps[b->off[sa]], &b->coefs[b->off[sa]], b->l[sb],
                    b->k[sb], &b->xyz[3 * sb], &b->exps[b->off[sb]], &b->coefs[b->off[sb]]);
}

double q_aux(const lx3c_basis* b, int s) { return q_aux_raw(b->l[s], b->k[s], &b->exps[b->off[s]], &b->coefs[b->off[s]]); }

// The estimate Q_ab Q_P is not a bound: on jittered clusters of the DF-J
// recipe the largest element of a triple reaches ~11x it (compact same-shell
// pairs).  A triple is kept when kSchwarzSafety Q_ab Q_P >= tol, so that the
// dropped triples stay below tol with that margin.
constexpr double kSchwarzSafety = 20.0;

struct DfjLaunch {
  ClassDesc desc;
  int grid = 1;
  // contraction at the (e 0|c) level (flag LX3C_DFJ_CONTRACT): the digest-5
  // descriptor, the bra-map pass (one sub-pair per tile, nC = nkrow) and its grid
  bool jeng = false;
  ClassDesc jdesc, mdesc;
  int mgrid = 1;
  double jflops = 0, pflops = 0;
  long long ntiles = 0;
  int4* d_sub = nullptr;
  int* d_prim = nullptr;
  int4* d_tiles = nullptr;
  std::vector<int4> sub;   // host copy of the sub-pair list (re-tiling)
  int kmax = 0;
};

struct DfjGroup {
  int la, lb, lc, Ka, Kb, Kc;
  std::vector<int32_t> pairs, auxs, counts;
  long long ntasks = 0;
  double flops = 0, nint = 0;
  int32_t* d_pairs = nullptr;
  int32_t* d_auxs = nullptr;
  int4* d_pair_ao = nullptr;
  int* d_aux_ao = nullptr;
  double* d_pairrec = nullptr;
  double* d_pairab = nullptr;
  double* d_auxrec = nullptr;
  double* d_auxc = nullptr;
  DfjLaunch L[2];
  // gradient: derivative classes (centre 0: (la+1,lb) scaled, (la-1,lb);
  // centre 1: (la,lb+1) scaled, (la,lb-1)), each with two orientations
  struct Deriv {
    int centre, plus, l1, l2;
    DfjLaunch L[2];
    int4* d_gmap = nullptr;
  };
  std::vector<Deriv> deriv;
  int2* d_pair_atoms = nullptr;
  int* d_aux_atom = nullptr;
  double gflops = 0;
};

// Derivative map for one derivative class (see ClassDesc::gmap).
std::vector<int4> derivative_map(int la, int lb, int centre, int plus, int gstart[4], int& nmax) {
  std::vector<std::vector<int4>> byax(3);
  const int l1 = la + (centre == 0 ? (plus ? 1 : -1) : 0), l2 = lb + (centre == 1 ? (plus ? 1 : -1) : 0);
  const int ncB = ncart(lb);
  auto carts = [](int l) {
    std::vector<std::array<int, 3>> v;
    for (int x = l; x >= 0; --x)
      for (int y = l - x; y >= 0; --y) v.push_back({x, y, l - x - y});
    return v;
  };
  auto c1 = carts(l1), c2 = carts(l2);
  for (size_t i1 = 0; i1 < c1.size(); ++i1)
    for (size_t i2 = 0; i2 < c2.size(); ++i2)
      for (int ax = 0; ax < 3; ++ax) {
        std::array<int, 3> a = c1[i1], b = c2[i2];
        std::array<int, 3>& moved = centre == 0 ? a : b;
        int factor;
        if (plus) {  // (x + 1_ax) present in the block: original x = moved - 1_ax
          if (moved[ax] < 1) continue;
          moved[ax] -= 1;
          factor = 1;
        } else {     // (x - 1_ax) in the block: original x = moved + 1_ax, factor -x_ax
          moved[ax] += 1;
          factor = -moved[ax];
        }
        const int ia = cart_index(a[0], a[1], a[2]), ib = cart_index(b[0], b[1], b[2]);
        byax[ax].push_back(int4{(int)i1, (int)i2, ia * ncB + ib, factor});
      }
  std::vector<int4> out;
  nmax = 0;
  for (int ax = 0; ax < 3; ++ax) {
    gstart[ax] = (int)out.size();
    out.insert(out.end(), byax[ax].begin(), byax[ax].end());
    nmax = std::max(nmax, (int)byax[ax].size());
  }
  gstart[3] = (int)out.size();
  return out;
}

}  // namespace

struct lx3c_dfj {
  const lx3c_basis* orb = nullptr;
  const lx3c_basis* aux = nullptr;
  long long nao = 0, naux_ao = 0;
  double tol = 0;
  int natom = 0;
  bool gradient = false;
  std::vector<DfjGroup> groups;
  double* d_sph = nullptr;          // solid-harmonic matrices for l = 0..7
  std::vector<int> sph_off;
  // exact fixed-point accumulators (two words per element): gamma, J, gradient
  unsigned long long* d_gacc = nullptr;
  unsigned long long* d_Jacc = nullptr;
  unsigned long long* d_facc = nullptr;
  // (e 0|c)-level contraction: bra maps, D through M^T and y, sized for the
  // largest launch and reused launch after launch
  bool contract = false;
  double* d_jM = nullptr;
  double* d_jD = nullptr;
  unsigned long long* d_jY = nullptr;
};

namespace lx3c {
const lx3c_basis* dfj_orbital_basis(const lx3c_dfj* plan) { return plan->orb; }
}  // namespace lx3c

extern "C" {

void lx3c_dfj_destroy(lx3c_dfj* p) {
  if (!p) return;
  for (auto& g : p->groups) {
    cudaFree(g.d_pairs); cudaFree(g.d_auxs); cudaFree(g.d_pair_ao); cudaFree(g.d_aux_ao);
    cudaFree(g.d_pairrec); cudaFree(g.d_pairab); cudaFree(g.d_auxrec); cudaFree(g.d_auxc);
    for (auto& L : g.L) {
      cudaFree(L.d_sub); cudaFree(L.d_prim); cudaFree(L.d_tiles);
    }
    for (auto& dv : g.deriv) {
      cudaFree(dv.d_gmap);
      for (auto& L : dv.L) {
        cudaFree(L.d_sub); cudaFree(L.d_prim); cudaFree(L.d_tiles);
      }
    }
    cudaFree(g.d_pair_atoms); cudaFree(g.d_aux_atom);
  }
  cudaFree(p->d_sph);
  cudaFree(p->d_gacc);
  cudaFree(p->d_Jacc);
  cudaFree(p->d_facc);
  cudaFree(p->d_jM);
  cudaFree(p->d_jD);
  cudaFree(p->d_jY);
  delete p;
}

lx3c_status lx3c_dfj_plan(lx3c_dfj** out, const lx3c_basis* orb, const lx3c_basis* aux, double schwarz_tol,
                          int flags, void* stream) {
  if (!out) return dfail(LX3C_EINVAL, "null output pointer");
  *out = nullptr;
  if (!orb || !aux) return dfail(LX3C_EINVAL, "null basis");
  if (orb->nshell <= 0 || aux->nshell <= 0) return dfail(LX3C_EINVAL, "empty basis");
  if (!(schwarz_tol >= 0.0)) return dfail(LX3C_EINVAL, "negative or NaN tolerance");
  const bool want_grad = (flags & 1) != 0;
  const bool contract = (flags & 2) != 0;
  for (int64_t s = 0; s < orb->nshell; ++s)
    if (orb->l[s] > LX3C_LMAX_ORB - (want_grad ? 1 : 0))
      return dfail(LX3C_ENOTSUP, "orbital shell beyond the supported l");
  if (want_grad) {
    for (int64_t s = 0; s < orb->nshell; ++s)
      if (orb->atom[s] < 0) return dfail(LX3C_EINVAL, "gradient needs an atom index on every shell");
    for (int64_t s = 0; s < aux->nshell; ++s)
      if (aux->atom[s] < 0) return dfail(LX3C_EINVAL, "gradient needs an atom index on every shell");
  }
  DevState* ds;
  int rc = device_state_get(&ds);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  std::unique_ptr<lx3c_dfj> p(new lx3c_dfj);
  p->orb = orb;
  p->aux = aux;
  p->tol = schwarz_tol;
  std::vector<int> ao(orb->nshell + 1, 0), aq(aux->nshell + 1, 0);
  for (int64_t s = 0; s < orb->nshell; ++s) ao[s + 1] = ao[s] + 2 * orb->l[s] + 1;
  for (int64_t s = 0; s < aux->nshell; ++s) aq[s + 1] = aq[s] + 2 * aux->l[s] + 1;
  p->nao = ao[orb->nshell];
  p->naux_ao = aq[aux->nshell];
  p->gradient = want_grad;
  for (int64_t s = 0; s < orb->nshell; ++s) p->natom = std::max(p->natom, orb->atom[s] + 1);
  for (int64_t s = 0; s < aux->nshell; ++s) p->natom = std::max(p->natom, aux->atom[s] + 1);
  // ket shells by (l, K), sorted by decreasing Q_P
  std::map<std::pair<int, int>, std::vector<std::pair<double, int>>> kets;
  for (int64_t s = 0; s < aux->nshell; ++s) kets[{aux->l[s], aux->k[s]}].push_back({q_aux(aux, (int)s), (int)s});
  for (auto& kv : kets)
    std::sort(kv.second.begin(), kv.second.end(), [](auto& x, auto& y) { return x.first > y.first || (x.first == y.first && x.second < y.second); });
  // unique shell pairs, canonical orientation (l, K) of the first >= second
  std::map<std::tuple<int, int, int, int>, std::vector<std::pair<int, int>>> bra;
  std::map<std::tuple<int, int, int, int>, std::vector<double>> braq;
  for (int a = 0; a < (int)orb->nshell; ++a)
    for (int b = a; b < (int)orb->nshell; ++b) {
      int s1 = a, s2 = b;
      if (std::make_pair(orb->l[s1], orb->k[s1]) < std::make_pair(orb->l[s2], orb->k[s2])) std::swap(s1, s2);
      auto key = std::make_tuple(orb->l[s1], orb->k[s1], orb->l[s2], orb->k[s2]);
      bra[key].push_back({s1, s2});
      braq[key].push_back(q_pair(orb, s1, s2));
    }
  for (auto& bk : bra) {
    const auto& pl = bk.second;
    const auto& ql = braq[bk.first];
    for (auto& kk : kets) {
      DfjGroup g;
      g.la = std::get<0>(bk.first); g.Ka = std::get<1>(bk.first);
      g.lb = std::get<2>(bk.first); g.Kb = std::get<3>(bk.first);
      g.lc = kk.first.first; g.Kc = kk.first.second;
      const auto& kl = kk.second;
      for (auto& e : kl) g.auxs.push_back(e.second);
      for (size_t i = 0; i < pl.size(); ++i) {
        const double thr = ql[i] > 0 ? schwarz_tol / (kSchwarzSafety * ql[i]) : 1e308;
        // number of ket shells with Q_P >= thr (prefix of the sorted list)
        int lo = 0, hi = (int)kl.size();
        while (lo < hi) {
          int mid = (lo + hi) / 2;
          if (kl[mid].first >= thr) lo = mid + 1; else hi = mid;
        }
        if (lo == 0) continue;
        g.pairs.push_back(pl[i].first);
        g.pairs.push_back(pl[i].second);
        g.counts.push_back(lo);
        g.ntasks += lo;
      }
      if (g.counts.empty()) continue;
      p->groups.push_back(std::move(g));
    }
  }
  // contributions per atom to the gradient's fixed-point accumulators
  std::vector<double> fadds(std::max(p->natom, 1), 0.0);
  // per group: orientation split, tiles, device lists
  for (auto& g : p->groups) {
    const long long np = (long long)g.counts.size(), na = (long long)g.auxs.size();
    const int nbra = (2 * g.la + 1) * (2 * g.lb + 1), nket = 2 * g.lc + 1;
    g.nint = (double)nbra * nket * (double)g.ntasks;
    std::vector<int4> sub[2];
    std::vector<int> prim[2];
    int kmax[2] = {0, 0}, cmax = 0;
    for (long long i = 0; i < np; ++i) {
      int oa = (int)prim[0].size(), ob = (int)prim[1].size();
      split_orientation(orb, g.pairs[2 * i], g.pairs[2 * i + 1], g.la, g.lb, prim[0], prim[1]);
      int na_ = (int)prim[0].size() - oa, nb_ = (int)prim[1].size() - ob;
      if (na_) sub[0].push_back(int4{(int)i, oa, na_, 0});
      if (nb_) sub[1].push_back(int4{(int)i, ob, nb_, 0});
      kmax[0] = std::max(kmax[0], na_);
      kmax[1] = std::max(kmax[1], nb_);
      cmax = std::max(cmax, g.counts[i]);
    }
    std::vector<int4> pao(np);
    std::vector<int> aao(na);
    for (long long i = 0; i < np; ++i)
      pao[i] = int4{ao[g.pairs[2 * i]], ao[g.pairs[2 * i + 1]], g.pairs[2 * i] == g.pairs[2 * i + 1] ? 1 : 0, 0};
    for (long long q = 0; q < na; ++q) aao[q] = aq[g.auxs[q]];
    const int Kab = g.Ka * g.Kb;
    DCUDA(cudaMalloc(&g.d_pairs, np * 8));
    DCUDA(cudaMalloc(&g.d_auxs, na * 4));
    DCUDA(cudaMalloc(&g.d_pair_ao, np * sizeof(int4)));
    DCUDA(cudaMalloc(&g.d_aux_ao, na * 4));
    DCUDA(cudaMalloc(&g.d_pairrec, (size_t)np * Kab * kPairRec * 8));
    DCUDA(cudaMalloc(&g.d_pairab, (size_t)np * 3 * 8));
    DCUDA(cudaMalloc(&g.d_auxrec, (size_t)na * g.Kc * kAuxRec * 8));
    DCUDA(cudaMalloc(&g.d_auxc, (size_t)na * 3 * 8));
    DCUDA(cudaMemcpyAsync(g.d_pairs, g.pairs.data(), np * 8, cudaMemcpyHostToDevice, st));
    DCUDA(cudaMemcpyAsync(g.d_auxs, g.auxs.data(), na * 4, cudaMemcpyHostToDevice, st));
    DCUDA(cudaMemcpyAsync(g.d_pair_ao, pao.data(), np * sizeof(int4), cudaMemcpyHostToDevice, st));
    DCUDA(cudaMemcpyAsync(g.d_aux_ao, aao.data(), na * 4, cudaMemcpyHostToDevice, st));
    for (int o = 0; o < 2; ++o) {
      if (sub[o].empty()) continue;
      DfjLaunch& L = g.L[o];
      const ClassTables* ct;
      try {
        ct = &class_tables(o ? g.lb : g.la, o ? g.la : g.lb, g.lc, 1);
      } catch (std::exception& e) {
        return dfail(LX3C_ENOTSUP, e.what());
      }
      DevClass* dc;
      rc = device_class_get(ds, *ct, &dc);
      if (rc) return rc;
      ClassDesc& d = L.desc;
      if (fill_class_desc(d, *ct, *dc, ds, o, kmax[o], Kab, g.Kc, fill_bound(sub[o], g.counts, cmax)) < 0)
        return dfail(LX3C_ENOTSUP, "class does not fit in shared memory");
      {
        // executed flops: each sub-pair's primitive pairs through this
        // orientation's primitive stages, its contracted stages and the
        // digestion (4 flops per integral) once per kept ket shell
        double tris = 0, primtris = 0;
        for (auto& sp : sub[o]) {
          tris += g.counts[sp.x];
          primtris += (double)g.counts[sp.x] * sp.z * g.Kc;
        }
        g.flops += primtris * ct->flops_prim + tris * (ct->flops_contr + 4.0 * nbra * nket);
      }
      std::vector<int4> tiles;
      for (size_t s = 0; s < sub[o].size(); ++s) {
        const int cnt = g.counts[sub[o][s].x];
        for (int a0 = 0; a0 < cnt; a0 += d.T) tiles.push_back(int4{(int)s, a0, std::min(d.T, cnt - a0), 0});
      }
      L.ntiles = (long long)tiles.size();
      L.sub = sub[o];
      L.kmax = kmax[o];
      DCUDA(cudaMalloc(&L.d_sub, sub[o].size() * sizeof(int4)));
      DCUDA(cudaMalloc(&L.d_prim, std::max<size_t>(prim[o].size(), 1) * sizeof(int)));
      DCUDA(cudaMalloc(&L.d_tiles, tiles.size() * sizeof(int4)));
      DCUDA(cudaMemcpyAsync(L.d_sub, sub[o].data(), sub[o].size() * sizeof(int4), cudaMemcpyHostToDevice, st));
      DCUDA(cudaMemcpyAsync(L.d_prim, prim[o].data(), prim[o].size() * sizeof(int), cudaMemcpyHostToDevice, st));
      DCUDA(cudaMemcpyAsync(L.d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
      d.npair = np;
      d.naux = na;
      d.nsub = (long long)sub[o].size();
      d.ntiles = L.ntiles;
      d.ntile_aux = 1;
      d.tiles = L.d_tiles;
      d.subpairs = L.d_sub;
      d.primidx = L.d_prim;
      d.pairrec = g.d_pairrec; d.pairab = g.d_pairab; d.auxrec = g.d_auxrec; d.auxc = g.d_auxc;
      d.digest = 1;
      set_digest_scratch(d);
      if ((long long)d.smem_doubles * 8 > 232448) return dfail(LX3C_ENOTSUP, "digestion scratch does not fit");
      d.ldD = p->nao;
      d.pair_ao = g.d_pair_ao;
      d.aux_ao = g.d_aux_ao;
      const int occ = eri3c_occupancy(d.smem_doubles * 8);
      L.grid = (int)std::min<long long>(L.ntiles, (long long)dev_nsm(ds) * occ * 8);
      if (contract) {
        // the bra-map pass: the class stages with nC = nkrow, one sub-pair per tile
        ClassTables ctm = *ct;
        ctm.nC = ct->nkrow;
        ctm.NV = ctm.NW = ctm.NF = ctm.NACC = 0;
        ctm.ncc = 0;
        LaunchShape shm{1, 1, 1, 0};
        ClassDesc dm;
        fill_desc_common(dm, ctm, *dc, dev_boys_tab(ds), dev_boys_mid(ds), o, kmax[o], Kab, g.Kc, shm);
        ClassDesc dj = d;
        dj.digest = 5;
        {
          // the gather output (X region) is live in this epilogue; the P
          // accumulators before it (Y region) are dead after the gather
          const long long need = ct->nkrow + 2LL * dj.T * ct->ncc;
          if (need <= (long long)dj.V.base - dj.P.base) {
            dj.dscr = dj.P.base;
          } else {
            dj.dscr = dj.smem_doubles;
            dj.smem_doubles += (int)need;
          }
        }
        // flops: per triple the primitive loop, the gather and the two
        // contractions over (e, c) (plus gamma's ket transform); per sub-pair
        // the bra map (the HRR and bra stages at nC = nkrow) and two GEMVs
        const double gather = 2.0 * ct->gterm.size(), ket = 2.0 * ct->kent.size() * ct->nkrow;
        const double hrrbra = (ct->flops_contr - gather - ket) / ct->nC * ct->nkrow;
        const double nab = (double)d.onA * d.onB, nk = ct->nkrow;
        double tris = 0, primtris = 0;
        for (auto& sp : sub[o]) {
          tris += g.counts[sp.x];
          primtris += (double)g.counts[sp.x] * sp.z * g.Kc;
        }
        const double jflops = primtris * ct->flops_prim + tris * (gather + 4.0 * nk * ct->ncc + 2.0 * ct->kent.size()) +
                              (double)d.nsub * (hrrbra + 4.0 * nab * nk);
        // the same triples digested per integral (what the plain path counts)
        const double pflops = primtris * ct->flops_prim + tris * (ct->flops_contr + 4.0 * nab * ct->nC);
        // contract the launch only where that saves work: with few kets per
        // pair the per-pair bra maps cost more than the per-triple stages
        // they replace
        if ((long long)dm.smem_doubles * 8 <= 232448 && (long long)dj.smem_doubles * 8 <= 232448 &&
            jflops < pflops) {
          dm.npair = np; dm.naux = na; dm.nsub = d.nsub; dm.subpairs = d.subpairs; dm.pairab = g.d_pairab;
          L.jeng = true;
          L.mdesc = dm;
          L.jdesc = dj;
          L.mgrid = (int)std::min<long long>(d.nsub, (long long)dev_nsm(ds) * 4);
          L.jflops = jflops;
          L.pflops = pflops;
          p->contract = true;
        }
      }
    }
    if (!want_grad) continue;
    // ---- gradient launches
    std::vector<int2> pat(np);
    std::vector<int> aat(na);
    for (long long i = 0; i < np; ++i) pat[i] = int2{orb->atom[g.pairs[2 * i]], orb->atom[g.pairs[2 * i + 1]]};
    for (long long q = 0; q < na; ++q) aat[q] = aux->atom[g.auxs[q]];
    DCUDA(cudaMalloc(&g.d_pair_atoms, np * sizeof(int2)));
    DCUDA(cudaMalloc(&g.d_aux_atom, na * 4));
    DCUDA(cudaMemcpyAsync(g.d_pair_atoms, pat.data(), np * sizeof(int2), cudaMemcpyHostToDevice, st));
    DCUDA(cudaMemcpyAsync(g.d_aux_atom, aat.data(), na * 4, cudaMemcpyHostToDevice, st));
    std::vector<double> gket_on_atom(p->natom, 0.0);
    for (long long q = 0; q < na; ++q)
      if (aat[q] >= 0) gket_on_atom[aat[q]] += 1.0;
    for (int centre = 0; centre < 2; ++centre)
      for (int plus = 1; plus >= 0; --plus) {
        const int l1 = g.la + (centre == 0 ? (plus ? 1 : -1) : 0), l2 = g.lb + (centre == 1 ? (plus ? 1 : -1) : 0);
        if (l1 < 0 || l2 < 0) continue;
        DfjGroup::Deriv dv;
        dv.centre = centre; dv.plus = plus; dv.l1 = l1; dv.l2 = l2;
        int gst[4], nmax = 0;
        std::vector<int4> gmap = derivative_map(g.la, g.lb, centre, plus, gst, nmax);
        DCUDA(cudaMalloc(&dv.d_gmap, gmap.size() * sizeof(int4)));
        DCUDA(cudaMemcpyAsync(dv.d_gmap, gmap.data(), gmap.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
        std::vector<int4> dsub[2];
        std::vector<int> dprim[2];
        int dk[2] = {0, 0};
        for (long long i = 0; i < np; ++i) {
          int oa = (int)dprim[0].size(), ob = (int)dprim[1].size();
          split_orientation(orb, g.pairs[2 * i], g.pairs[2 * i + 1], l1, l2, dprim[0], dprim[1]);
          int na_ = (int)dprim[0].size() - oa, nb_ = (int)dprim[1].size() - ob;
          if (na_) dsub[0].push_back(int4{(int)i, oa, na_, 0});
          if (nb_) dsub[1].push_back(int4{(int)i, ob, nb_, 0});
          dk[0] = std::max(dk[0], na_);
          dk[1] = std::max(dk[1], nb_);
        }
        for (int o = 0; o < 2; ++o) {
          if (dsub[o].empty()) continue;
          DfjLaunch& L = dv.L[o];
          const ClassTables* ct;
          try {
            ct = &class_tables(o ? l2 : l1, o ? l1 : l2, g.lc, 0);
          } catch (std::exception& e) {
            return dfail(LX3C_ENOTSUP, e.what());
          }
          DevClass* dc;
          rc = device_class_get(ds, *ct, &dc);
          if (rc) return rc;
          ClassDesc& d = L.desc;
          if (fill_class_desc(d, *ct, *dc, ds, o, dk[o], Kab, g.Kc, fill_bound(dsub[o], g.counts, cmax)) < 0)
            return dfail(LX3C_ENOTSUP, "derivative class does not fit in shared memory");
          {
            // executed flops of this derivative launch (as for the class
            // launches) plus its contraction with D, c (2 flops per entry of
            // the derivative map and ket function)
            double tris = 0, primtris = 0;
            for (auto& sp : dsub[o]) {
              tris += g.counts[sp.x];
              primtris += (double)g.counts[sp.x] * sp.z * g.Kc;
            }
            g.gflops += primtris * ct->flops_prim + tris * (ct->flops_contr + 2.0 * gmap.size() * (2 * g.lc + 1));
          }
          // entries per partial sum: balances the partial's FMA chain (E (nC+1))
          // against the final sum over the nmax / E partials of an axis
          const int E = std::max(1, std::min(32, (int)std::lround(std::sqrt((double)nmax / (d.nC + 1)))));
          const int nch = std::max(1, (nmax + E - 1) / E);
          const int nAp = 2 * g.la + 1, ncA = ncart(g.la), nBp = 2 * g.lb + 1, ncB = ncart(g.lb);
          d.g_echunk = E;
          d.g_base = place_epilogue_scratch(d, nAp * ncB + ncA * ncB + (long long)d.T * 3 * (nch + 1));
          if (d.smem_doubles * 8 > 232448) return dfail(LX3C_ENOTSUP, "gradient epilogue does not fit");
          d.g_centre = centre;
          d.g_nAp = nAp; d.g_ncA = ncA; d.g_nBp = nBp; d.g_ncB = ncB; d.g_nch = nch;
          for (int k = 0; k < 4; ++k) d.gstart[k] = gst[k];
          d.gmap = dv.d_gmap;
          std::vector<int4> tiles;
          for (size_t s2 = 0; s2 < dsub[o].size(); ++s2) {
            const int pi = dsub[o][s2].x, cnt = g.counts[pi];
            const int tat = orb->atom[g.pairs[2 * pi + centre]];
            for (int a0 = 0; a0 < cnt; a0 += d.T) {
              tiles.push_back(int4{(int)s2, a0, std::min(d.T, cnt - a0), 0});
              if (tat >= 0) fadds[tat] += 1.0;  // one add per axis per tile
            }
          }
          // one add per triple to the ket shell's atom: at most this
          // launch's sub-pairs times the group's kets on that atom
          for (int a = 0; a < p->natom; ++a) fadds[a] += (double)dsub[o].size() * gket_on_atom[a];
          L.ntiles = (long long)tiles.size();
          DCUDA(cudaMalloc(&L.d_sub, dsub[o].size() * sizeof(int4)));
          DCUDA(cudaMalloc(&L.d_prim, std::max<size_t>(dprim[o].size(), 1) * sizeof(int)));
          DCUDA(cudaMalloc(&L.d_tiles, tiles.size() * sizeof(int4)));
          DCUDA(cudaMemcpyAsync(L.d_sub, dsub[o].data(), dsub[o].size() * sizeof(int4), cudaMemcpyHostToDevice, st));
          DCUDA(cudaMemcpyAsync(L.d_prim, dprim[o].data(), dprim[o].size() * sizeof(int), cudaMemcpyHostToDevice, st));
          DCUDA(cudaMemcpyAsync(L.d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
          d.npair = np; d.naux = na;
          d.nsub = (long long)dsub[o].size();
          d.ntiles = L.ntiles;
          d.ntile_aux = 1;
          d.tiles = L.d_tiles; d.subpairs = L.d_sub; d.primidx = L.d_prim;
          d.pairrec = g.d_pairrec; d.pairab = g.d_pairab; d.auxrec = g.d_auxrec; d.auxc = g.d_auxc;
          d.digest = 2;
          d.ldD = p->nao;
          d.pair_ao = g.d_pair_ao; d.aux_ao = g.d_aux_ao;
          d.pair_atoms = g.d_pair_atoms; d.aux_atom = g.d_aux_atom;
          const int occ = eri3c_occupancy(d.smem_doubles * 8);
          L.grid = (int)std::min<long long>(L.ntiles, (long long)dev_nsm(ds) * occ * 8);
        }
        g.deriv.push_back(dv);
      }
  }
  if (want_grad && *std::max_element(fadds.begin(), fadds.end()) >= kFixMaxAdds)
    return dfail(LX3C_ENOTSUP, "gradient: an atom's force accumulator would take 2^32 or more contributions");
  if (want_grad) {
    std::vector<double> sph;
    p->sph_off.assign(9, 0);
    for (int l = 0; l <= 7; ++l) {
      auto T = solid_matrix(l);
      p->sph_off[l] = (int)sph.size();
      sph.insert(sph.end(), T.begin(), T.end());
    }
    p->sph_off[8] = (int)sph.size();
    DCUDA(cudaMalloc(&p->d_sph, sph.size() * 8));
    DCUDA(cudaMemcpyAsync(p->d_sph, sph.data(), sph.size() * 8, cudaMemcpyHostToDevice, st));
    DCUDA(cudaStreamSynchronize(st));
    for (auto& g : p->groups)
      for (auto& dv : g.deriv)
        for (auto& L : dv.L) {
          L.desc.Ta = p->d_sph + p->sph_off[g.la];
          L.desc.Tb = p->d_sph + p->sph_off[g.lb];
        }
  }
  if (p->contract) {
    size_t nm = 1, nd = 1;
    for (auto& g : p->groups)
      for (auto& L : g.L)
        if (L.jeng) {
          nm = std::max(nm, (size_t)L.desc.nsub * L.desc.onA * L.desc.onB * L.mdesc.nkrow);
          nd = std::max(nd, (size_t)L.desc.nsub * L.mdesc.nkrow);
        }
    DCUDA(cudaMalloc(&p->d_jM, nm * 8));
    DCUDA(cudaMalloc(&p->d_jD, nd * 8));
    DCUDA(cudaMalloc(&p->d_jY, nd * kFixBytes));
    for (auto& g : p->groups)
      for (auto& L : g.L)
        if (L.jeng) {
          for (ClassDesc* d : {&L.mdesc, &L.jdesc}) {
            d->jM = p->d_jM;
            d->jD = p->d_jD;
            d->jY = p->d_jY;
          }
        }
  }
  DCUDA(cudaMalloc(&p->d_gacc, (size_t)p->naux_ao * kFixBytes));
  DCUDA(cudaMalloc(&p->d_Jacc, (size_t)p->nao * p->nao * kFixBytes));
  if (want_grad) DCUDA(cudaMalloc(&p->d_facc, (size_t)p->natom * 3 * kFixBytes));
  DCUDA(cudaStreamSynchronize(st));
  *out = p.release();
  return LX3C_OK;
}

lx3c_status lx3c_dfj_execute(lx3c_dfj* p, const double* D, const double* c, double* gamma, double* J, void* stream) {
  if (!p) return dfail(LX3C_EINVAL, "null plan");
  if (!D || !c || (!gamma && !J)) return dfail(LX3C_EINVAL, "null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  if (gamma) DCUDA(cudaMemsetAsync(p->d_gacc, 0, p->naux_ao * kFixBytes, st));
  if (J) DCUDA(cudaMemsetAsync(p->d_Jacc, 0, p->nao * p->nao * kFixBytes, st));
  for (auto& g : p->groups) {
    const long long np = (long long)g.counts.size(), na = (long long)g.auxs.size();
    DCUDA(launch_pair_precompute(p->orb->dev(), g.d_pairs, np, g.Ka, g.Kb, g.d_pairrec, g.d_pairab, st));
    DCUDA(launch_aux_precompute(p->aux->dev(), g.d_auxs, na, g.Kc, g.d_auxrec, g.d_auxc, st));
    for (auto& L : g.L) {
      if (!L.ntiles) continue;
      ClassDesc d = L.jeng ? L.jdesc : L.desc;
      d.D = D;
      d.cvec = c;
      d.gacc = gamma ? p->d_gacc : nullptr;
      d.Jacc = J ? p->d_Jacc : nullptr;
      if (L.jeng) {
        // bra maps, D through M^T, the tiles at the (e 0|c) level, then J = M y
        ClassDesc dm = L.mdesc;
        dm.D = D;
        dm.gacc = d.gacc;
        dm.Jacc = d.Jacc;
        dm.ldD = d.ldD;
        dm.pair_ao = d.pair_ao;
        if (J) DCUDA(cudaMemsetAsync(p->d_jY, 0, (size_t)d.nsub * d.nkrow * kFixBytes, st));
        DCUDA(launch_jeng_matrix(dm, L.mgrid, st));
        if (gamma) DCUDA(launch_jeng_pair(dm, 0, st));
        DCUDA(launch_eri3c(d, L.grid, st));
        if (J) DCUDA(launch_jeng_pair(dm, 1, st));
      } else {
        DCUDA(launch_eri3c(d, L.grid, st));
      }
    }
  }
  if (gamma) DCUDA(launch_fix_finish(p->d_gacc, p->naux_ao, gamma, st));
  if (J) DCUDA(launch_fix_finish_J(p->d_Jacc, p->nao, J, st));
  return LX3C_OK;
}

lx3c_status lx3c_dfj_execute_multi(lx3c_dfj* p, int nd, const double* D, const double* c, double* gamma, double* J,
                                   void* stream) {
  if (!p) return dfail(LX3C_EINVAL, "null plan");
  if (nd < 1 || nd > 8) return dfail(LX3C_EINVAL, "execute_multi: nd must be in 1..8");
  if ((gamma && !D) || (J && !c) || (!gamma && !J)) return dfail(LX3C_EINVAL, "execute_multi: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const long long dstride = p->nao * p->nao, cstride = p->naux_ao;
  // check every launch's scratch before launching anything
  std::vector<ClassDesc> descs;
  std::vector<int> grids;
  for (auto& g : p->groups)
    for (auto& L : g.L) {
      if (!L.ntiles) continue;
      ClassDesc d = L.desc;
      d.digest = 4;
      d.nd = nd;
      d.dstride = dstride;
      d.cstride = cstride;
      d.D = D;
      d.cvec = c;
      d.gamma = gamma;
      d.J = J;
      const long long kAB = ((long long)d.onA * d.onB + 3) & ~3LL, kR = ((long long)d.T * d.nC + 3) & ~3LL;
      d.dscr = place_epilogue_scratch(d, 8 * (kAB + kR));
      if ((long long)d.smem_doubles * 8 > 232448) return dfail(LX3C_ENOTSUP, "execute_multi: scratch does not fit");
      descs.push_back(d);
      grids.push_back(L.grid);
    }
  if (gamma) DCUDA(cudaMemsetAsync(gamma, 0, (size_t)nd * cstride * 8, st));
  if (J) DCUDA(cudaMemsetAsync(J, 0, (size_t)nd * dstride * 8, st));
  size_t li = 0;
  for (auto& g : p->groups) {
    const long long np = (long long)g.counts.size(), na = (long long)g.auxs.size();
    DCUDA(launch_pair_precompute(p->orb->dev(), g.d_pairs, np, g.Ka, g.Kb, g.d_pairrec, g.d_pairab, st));
    DCUDA(launch_aux_precompute(p->aux->dev(), g.d_auxs, na, g.Kc, g.d_auxrec, g.d_auxc, st));
    for (auto& L : g.L) {
      if (!L.ntiles) continue;
      DCUDA(launch_eri3c(descs[li], grids[li], st));
      ++li;
    }
  }
  if (J) {
    dim3 blk(32, 8), grd((unsigned)((p->nao + 31) / 32), (unsigned)((p->nao + 7) / 8));
    for (int k = 0; k < nd; ++k) symmetrize<<<grd, blk, 0, st>>>(J + k * dstride, p->nao);
    DCUDA(cudaGetLastError());
  }
  return LX3C_OK;
}

lx3c_status lx3c_dfj_energy(lx3c_dfj* p, const double* D, const double* c, double* gamma, double* energy,
                            void* stream) {
  if (!energy || !gamma) return dfail(LX3C_EINVAL, "null pointer");
  lx3c_status rc = lx3c_dfj_execute(p, D, c, gamma, nullptr, stream);
  if (rc) return rc;
  dot_energy<<<1, 256, 0, (cudaStream_t)stream>>>(c, gamma, p->naux_ao, energy);
  DCUDA(cudaGetLastError());
  return LX3C_OK;
}

lx3c_status lx3c_dfj_grad(lx3c_dfj* p, const double* D, const double* c, double* grad, void* stream) {
  if (!p) return dfail(LX3C_EINVAL, "null plan");
  if (!p->gradient) return dfail(LX3C_EINVAL, "plan was built without gradient support (flags & 1)");
  if (!D || !c || !grad) return dfail(LX3C_EINVAL, "null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  DCUDA(cudaMemsetAsync(p->d_facc, 0, (size_t)p->natom * 3 * kFixBytes, st));
  for (auto& g : p->groups) {
    const long long np = (long long)g.counts.size(), na = (long long)g.auxs.size();
    DCUDA(launch_aux_precompute(p->aux->dev(), g.d_auxs, na, g.Kc, g.d_auxrec, g.d_auxc, st));
    for (auto& dv : g.deriv) {
      DCUDA(launch_pair_precompute(p->orb->dev(), g.d_pairs, np, g.Ka, g.Kb, g.d_pairrec, g.d_pairab, st,
                                   dv.centre == 0 && dv.plus, dv.centre == 1 && dv.plus));
      for (auto& L : dv.L) {
        if (!L.ntiles) continue;
        ClassDesc d = L.desc;
        d.D = D;
        d.cvec = c;
        d.facc = p->d_facc;
        DCUDA(launch_eri3c(d, L.grid, st));
      }
    }
  }
  DCUDA(launch_fix_finish(p->d_facc, (long long)p->natom * 3, grad, st));
  return LX3C_OK;
}

lx3c_status lx3c_schwarz_pair(int la, int ka, const double* A, const double* ea, const double* ca, int lb, int kb,
                              const double* B, const double* eb, const double* cb, double* q) {
  if (!A || !ea || !ca || !B || !eb || !cb || !q || la < 0 || lb < 0 || ka < 1 || kb < 1)
    return dfail(LX3C_EINVAL, "schwarz_pair: bad argument");
  *q = kSchwarzSafety * q_pair_raw(la, ka, A, ea, ca, lb, kb, B, eb, cb);
  return LX3C_OK;
}

lx3c_status lx3c_schwarz_aux(int l, int k, const double* e, const double* c, double* q) {
  if (!e || !c || !q || l < 0 || k < 1) return dfail(LX3C_EINVAL, "schwarz_aux: bad argument");
  *q = q_aux_raw(l, k, e, c);
  return LX3C_OK;
}

lx3c_status lx3c_dfj_info(const lx3c_dfj* p, double* out, int n) {
  if (!p || (!out && n > 0)) return dfail(LX3C_EINVAL, "null pointer");
  double tasks = 0, nint = 0, flops = 0, launches = 2, gflops = 0, glaunches = p->gradient ? 1 : 0, slots = 0;
  for (auto& g : p->groups) {
    for (auto& L : g.L) {
      slots += (double)L.ntiles * L.desc.T;
      if (L.jeng) {
        flops += L.jflops - L.pflops;
        launches += 3;  // bra maps, D through M^T, J = M y
      }
    }
    tasks += (double)g.ntasks;
    nint += g.nint;
    flops += g.flops;
    gflops += g.gflops;
    launches += 2 + (g.L[0].ntiles > 0) + (g.L[1].ntiles > 0);
    if (p->gradient) glaunches += 1;
    for (auto& dv : g.deriv) glaunches += 1 + (dv.L[0].ntiles > 0) + (dv.L[1].ntiles > 0);
  }
  const double v[] = {(double)p->groups.size(), tasks, nint, flops, launches, (double)p->nao, (double)p->naux_ao,
                      (double)p->natom, gflops, glaunches, slots};
  for (int i = 0; i < n && i < 11; ++i) out[i] = v[i];
  return LX3C_OK;
}

lx3c_status lx3c_dfj_group(const lx3c_dfj* p, int gi, int32_t* info, int32_t* pairs, int32_t* counts,
                           int32_t* auxs) {
  if (!p) return dfail(LX3C_EINVAL, "null plan");
  if (gi < 0 || gi >= (int)p->groups.size()) return dfail(LX3C_EINVAL, "group index out of range");
  const DfjGroup& g = p->groups[gi];
  if (info) {
    const int32_t v[] = {g.la, g.lb, g.lc, g.Ka, g.Kb, g.Kc, (int32_t)g.counts.size(), (int32_t)g.auxs.size()};
    std::memcpy(info, v, sizeof(v));
  }
  if (pairs) std::memcpy(pairs, g.pairs.data(), g.pairs.size() * 4);
  if (counts) std::memcpy(counts, g.counts.data(), g.counts.size() * 4);
  if (auxs) std::memcpy(auxs, g.auxs.data(), g.auxs.size() * 4);
  return LX3C_OK;
}


}  // extern "C"

// ---------------------------------------------------------------------------
// Batched uneven workloads: several molecules' DF-J builds, every class mixed,
// as one persistent kernel captured in a CUDA graph (not in the paper).
// ---------------------------------------------------------------------------

namespace {

// Shape of one (class, orientation, kmax, Kc) launch: triples per tile T.
std::string shape_key(const ClassDesc& d) {
  char b[96];
  std::snprintf(b, sizeof(b), "%d,%d,%d,%d,%d,%d,%d", d.la, d.lb, d.lc, d.bra_pure, d.Kab, d.Kc, d.digest);
  return b;
}

// Re-tile one launch for triples-per-tile T (other shape fields recomputed by
// the planner for that T); returns false if T does not fit.
bool retile(DfjLaunch& L, const DfjGroup& g, const DevState* ds, int T) {
  const ClassTables& ct = class_tables(L.desc.la, L.desc.lb, L.desc.lc, L.desc.bra_pure);
  ClassDesc d = L.desc;
  const int mode = T >= 32 ? 0 : 1;
  // keep G from the planner's choice for this T
  LaunchShape sh = choose_shape(ct, L.kmax, d.Kc, T, dev_smem(ds));
  sh.T = T;
  sh.mode = mode;
  ClassDesc nd = d;
  fill_layout(nd, ct, sh);
  if (d.digest == 2) {
    nd.g_base = place_epilogue_scratch(nd, d.g_nAp * d.g_ncB + d.g_ncA * d.g_ncB + (long long)T * 3 * d.g_nch);
  } else if (d.digest == 1) {
    set_digest_scratch(nd);
  }
  if ((long long)nd.smem_doubles * 8 > 232448 - 64) return false;
  nd.nchunk = (nd.K + nd.G - 1) / nd.G;
  std::vector<int4> tiles;
  for (size_t s2 = 0; s2 < L.sub.size(); ++s2) {
    const int cnt = g.counts[L.sub[s2].x];
    for (int a0 = 0; a0 < cnt; a0 += T) tiles.push_back(int4{(int)s2, a0, std::min(T, cnt - a0), 0});
  }
  int4* dt = nullptr;
  if (cudaMalloc(&dt, tiles.size() * sizeof(int4)) != cudaSuccess) return false;
  cudaMemcpy(dt, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice);
  cudaFree(L.d_tiles);
  L.d_tiles = dt;
  L.ntiles = (long long)tiles.size();
  nd.tiles = dt;
  nd.ntiles = L.ntiles;
  L.desc = nd;
  const int occ = eri3c_occupancy(nd.smem_doubles * 8);
  L.grid = (int)std::min<long long>(L.ntiles, (long long)dev_nsm(ds) * occ * 8);
  return true;
}

}  // namespace

struct lx3c_batch {
  std::vector<lx3c_dfj*> mols;
  DevState* ds = nullptr;
  std::map<std::string, int> tuned;   // shape_key -> T
  int ntuned_measured = 0;
  // bound state
  ClassDesc* d_descs = nullptr;
  int2* d_work = nullptr;
  unsigned long long* d_counter = nullptr;  // one per tier
  long long nwork = 0;
  int ndesc = 0;
  int smem = 0;
  int grid = 0;
  // mode 1 splits the work items into occupancy tiers, each run by a
  // persistent kernel sized for the tier's largest item: items that fit three
  // CTAs per SM (the 40-register kernel), then two, then the rest
  struct Tier {
    long long off = 0, n = 0;
    int smem = 0, grid = 0, three = 0;
  };
  std::vector<Tier> tiers;
  cudaGraph_t graph = nullptr;        // mode 1: persistent kernels, one per tier
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph2 = nullptr;       // mode 2: class launches on parallel branches
  cudaGraphExec_t exec2 = nullptr;
  long long branch_kernels = 0;
  std::vector<const double*> D, c;
  std::vector<double*> gamma, J;
  long long plain_launches = 0, graph_kernels = 0;
};

namespace {

constexpr int kBranches = 4;

// Mode 2: the same build as a graph whose class launches (the one-class kernel,
// descriptor in the parameter space) are spread over kBranches parallel
// branches, longest first onto the least loaded branch; zeroing and
// precomputes come before the fork, J symmetrisation after the join.
cudaError_t capture_branches(lx3c_batch* b, const std::vector<ClassDesc>& descs, const std::vector<int>& grids,
                             const std::vector<std::pair<double, int>>& order, cudaStream_t cap) {
  if (b->exec2) { cudaGraphExecDestroy(b->exec2); b->exec2 = nullptr; }
  if (b->graph2) { cudaGraphDestroy(b->graph2); b->graph2 = nullptr; }
  cudaStream_t br[kBranches] = {};
  cudaEvent_t fork = nullptr, join[kBranches] = {};
  cudaError_t ce = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int i = 0; i < kBranches && ce == cudaSuccess; ++i) {
    ce = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
  }
  if (ce == cudaSuccess) ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (ce == cudaSuccess) {
    long long kernels = 0;
    const int nmol = (int)b->mols.size();
    for (int m = 0; m < nmol; ++m) {
      lx3c_dfj* p = b->mols[m];
      cudaMemsetAsync(p->d_gacc, 0, p->naux_ao * kFixBytes, cap);
      cudaMemsetAsync(p->d_Jacc, 0, p->nao * p->nao * kFixBytes, cap);
      for (auto& g : p->groups) {
        launch_pair_precompute(p->orb->dev(), g.d_pairs, (long long)g.counts.size(), g.Ka, g.Kb, g.d_pairrec,
                               g.d_pairab, cap);
        launch_aux_precompute(p->aux->dev(), g.d_auxs, (long long)g.auxs.size(), g.Kc, g.d_auxrec, g.d_auxc, cap);
        kernels += 2;
      }
    }
    cudaEventRecord(fork, cap);
    double load[kBranches] = {};
    for (int i = 0; i < kBranches; ++i) cudaStreamWaitEvent(br[i], fork, 0);
    for (auto& o : order) {
      int k = 0;
      for (int i = 1; i < kBranches; ++i)
        if (load[i] < load[k]) k = i;
      load[k] += o.first;
      launch_eri3c(descs[o.second], grids[o.second], br[k]);
      ++kernels;
    }
    for (int i = 0; i < kBranches; ++i) {
      cudaEventRecord(join[i], br[i]);
      cudaStreamWaitEvent(cap, join[i], 0);
    }
    for (int m = 0; m < nmol; ++m) {
      launch_fix_finish(b->mols[m]->d_gacc, b->mols[m]->naux_ao, b->gamma[m], cap);
      launch_fix_finish_J(b->mols[m]->d_Jacc, b->mols[m]->nao, b->J[m], cap);
      kernels += 2;
    }
    ce = cudaStreamEndCapture(cap, &b->graph2);
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&b->exec2, b->graph2, 0);
    b->branch_kernels = kernels;
  }
  for (int i = 0; i < kBranches; ++i) {
    if (br[i]) cudaStreamDestroy(br[i]);
    if (join[i]) cudaEventDestroy(join[i]);
  }
  if (fork) cudaEventDestroy(fork);
  return ce;
}

}  // namespace

extern "C" {

void lx3c_batch_destroy(lx3c_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->exec2) cudaGraphExecDestroy(b->exec2);
  if (b->graph2) cudaGraphDestroy(b->graph2);
  cudaFree(b->d_descs);
  cudaFree(b->d_work);
  cudaFree(b->d_counter);
  for (auto* m : b->mols) lx3c_dfj_destroy(m);
  delete b;
}

lx3c_status lx3c_batch_plan(lx3c_batch** out, int nmol, const lx3c_basis* const* orbs, const lx3c_basis* const* auxs,
                            double schwarz_tol, const char* tune_cache, void* stream) {
  if (!out) return dfail(LX3C_EINVAL, "null output pointer");
  *out = nullptr;
  if (nmol <= 0 || !orbs || !auxs) return dfail(LX3C_EINVAL, "empty molecule list");
  std::unique_ptr<lx3c_batch> b(new lx3c_batch);
  int rc = device_state_get(&b->ds);
  if (rc) return rc;
  for (int m = 0; m < nmol; ++m) {
    lx3c_dfj* p = nullptr;
    rc = lx3c_dfj_plan(&p, orbs[m], auxs[m], schwarz_tol, 0, stream);
    if (rc) return rc;
    b->mols.push_back(p);
  }
  // ---- autotuner: triples per tile for each launch signature, timed on the
  // signature's largest launch; results cached as "key T" lines.
  std::map<std::string, int> cache;
  if (tune_cache && *tune_cache) {
    std::ifstream f(tune_cache);
    std::string k;
    int T;
    while (f >> k >> T) cache[k] = T;
  }
  std::map<std::string, std::pair<DfjLaunch*, DfjGroup*>> biggest;
  for (auto* p : b->mols)
    for (auto& g : p->groups)
      for (auto& L : g.L) {
        if (!L.ntiles) continue;
        const std::string k = shape_key(L.desc);
        auto it = biggest.find(k);
        long long work = (long long)L.desc.T * L.ntiles;
        if (it == biggest.end() || (long long)it->second.first->desc.T * it->second.first->ntiles < work)
          biggest[k] = {&L, &g};
      }
  cudaStream_t st = (cudaStream_t)stream;
  double *tg = nullptr, *tJ = nullptr, *tD = nullptr, *tc = nullptr;
  bool measured = false;
  for (auto& kv : biggest) {
    if (cache.count(kv.first)) {
      b->tuned[kv.first] = cache[kv.first];
      continue;
    }
    DfjLaunch& L = *kv.second.first;
    DfjGroup& g = *kv.second.second;
    lx3c_dfj* owner = nullptr;
    for (auto* p : b->mols)
      for (auto& gg : p->groups)
        if (&gg == &g) owner = p;
    if (!tg) {
      long long mx = 0, mxa = 0;
      for (auto* p : b->mols) { mx = std::max(mx, p->nao); mxa = std::max(mxa, p->naux_ao); }
      DCUDA(cudaMalloc(&tg, mxa * kFixBytes)); DCUDA(cudaMalloc(&tc, mxa * 8));
      DCUDA(cudaMalloc(&tJ, mx * mx * kFixBytes)); DCUDA(cudaMalloc(&tD, mx * mx * 8));
      DCUDA(cudaMemset(tg, 0, mxa * kFixBytes)); DCUDA(cudaMemset(tJ, 0, mx * mx * kFixBytes));
      DCUDA(cudaMemset(tc, 0, mxa * 8)); DCUDA(cudaMemset(tD, 0, mx * mx * 8));
    }
    DCUDA(launch_pair_precompute(owner->orb->dev(), g.d_pairs, (long long)g.counts.size(), g.Ka, g.Kb, g.d_pairrec,
                                 g.d_pairab, st));
    DCUDA(launch_aux_precompute(owner->aux->dev(), g.d_auxs, (long long)g.auxs.size(), g.Kc, g.d_auxrec, g.d_auxc, st));
    const int T0 = L.desc.T;
    std::vector<int> cands = {T0};
    if (T0 >= 2) cands.push_back(T0 / 2);
    if (T0 <= 256) cands.push_back(T0 * 2);
    float best = 1e30f;
    int bestT = T0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // time every candidate on the same prefix of sub-pairs: about 8 waves of
    // the planner's tiles, the same triples whatever T is
    long long nsub_t = (long long)L.sub.size();
    {
      const long long cap = 8LL * dev_nsm(b->ds) * 2;
      long long nt = 0;
      for (long long s2 = 0; s2 < (long long)L.sub.size(); ++s2) {
        nt += (g.counts[L.sub[s2].x] + T0 - 1) / T0;
        if (nt >= cap) { nsub_t = s2 + 1; break; }
      }
    }
    for (int T : cands) {
      if (!retile(L, g, b->ds, T)) continue;
      ClassDesc d = L.desc;
      d.D = tD; d.cvec = tc;
      d.gacc = (unsigned long long*)tg; d.Jacc = (unsigned long long*)tJ;
      long long nt = 0;
      for (long long s2 = 0; s2 < nsub_t; ++s2) nt += (g.counts[L.sub[s2].x] + T - 1) / T;
      d.ntiles = nt;
      const int grid = (int)std::min<long long>(nt, L.grid);
      launch_eri3c(d, grid, st);
      cudaEventRecord(e0, st);
      launch_eri3c(d, grid, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bestT = T; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuned[kv.first] = bestT;
    cache[kv.first] = bestT;
    measured = true;
    ++b->ntuned_measured;
  }
  cudaFree(tg); cudaFree(tJ); cudaFree(tD); cudaFree(tc);
  // apply the tuned shapes to every launch
  for (auto* p : b->mols)
    for (auto& g : p->groups)
      for (auto& L : g.L) {
        if (!L.ntiles) continue;
        auto it = b->tuned.find(shape_key(L.desc));
        if (it != b->tuned.end() && it->second != L.desc.T) retile(L, g, b->ds, it->second);
      }
  if (measured && tune_cache && *tune_cache) {
    std::ofstream f(tune_cache);
    for (auto& kv : cache) f << kv.first << " " << kv.second << "\n";
  }
  DCUDA(cudaGetLastError());
  DCUDA(cudaStreamSynchronize(st));
  *out = b.release();
  return LX3C_OK;
}

lx3c_status lx3c_batch_bind(lx3c_batch* b, const double* const* D, const double* const* c, double* const* gamma,
                            double* const* J, void* stream) {
  if (!b || !D || !c || !gamma || !J) return dfail(LX3C_EINVAL, "null pointer");
  const int nmol = (int)b->mols.size();
  b->D.assign(D, D + nmol); b->c.assign(c, c + nmol);
  b->gamma.assign(gamma, gamma + nmol); b->J.assign(J, J + nmol);
  // descriptors with this binding's pointers, and the longest-first work list
  std::vector<ClassDesc> descs;
  std::vector<int> grids;
  std::vector<std::pair<double, int>> order;
  int smem = 0;
  b->plain_launches = 0;
  for (int m = 0; m < nmol; ++m) {
    lx3c_dfj* p = b->mols[m];
    b->plain_launches += 2;
    for (auto& g : p->groups) {
      b->plain_launches += 2;
      for (auto& L : g.L) {
        if (!L.ntiles) continue;
        ++b->plain_launches;
        ClassDesc d = L.desc;
        d.D = D[m]; d.cvec = c[m]; d.gacc = p->d_gacc; d.Jacc = p->d_Jacc;
        double fl = 0;
        lx3c_class_flops(d.la, d.lb, d.lc, d.Kab, d.Kc, 1, &fl);
        order.push_back({fl * (double)d.T * (double)L.ntiles, (int)descs.size()});
        descs.push_back(d);
        grids.push_back(L.grid);
        smem = std::max(smem, d.smem_doubles * 8);
      }
    }
  }
  std::stable_sort(order.begin(), order.end(), [](auto& x, auto& y) { return x.first > y.first; });
  // tiers: the items whose shared memory lets the 40-register persistent
  // kernel keep three CTAs per SM, then those that fit two CTAs of the
  // unrestricted one, then the others; longest first within each tier
  std::vector<int2> work;
  b->tiers.clear();
  auto tier_of = [&](int sm) { return persistent_occupancy(sm, 1) >= 3 ? 0 : (persistent_occupancy(sm, 0) >= 2 ? 1 : 2); };
  for (int tier = 0; tier < 3; ++tier) {
    lx3c_batch::Tier T;
    T.off = (long long)work.size();
    T.three = tier == 0 ? 1 : 0;
    for (auto& o : order) {
      const int sm = descs[o.second].smem_doubles * 8;
      if (tier_of(sm) != tier) continue;
      T.smem = std::max(T.smem, sm);
      for (long long t = 0; t < descs[o.second].ntiles; ++t) work.push_back(int2{o.second, (int)t});
    }
    T.n = (long long)work.size() - T.off;
    if (!T.n) continue;
    T.grid = dev_nsm(b->ds) * persistent_occupancy(T.smem, T.three);
    b->tiers.push_back(T);
  }
  cudaFree(b->d_descs);
  cudaFree(b->d_work);
  if (!b->d_counter) DCUDA(cudaMalloc(&b->d_counter, 3 * sizeof(unsigned long long)));
  DCUDA(cudaMalloc(&b->d_descs, descs.size() * sizeof(ClassDesc)));
  DCUDA(cudaMalloc(&b->d_work, std::max<size_t>(work.size(), 1) * sizeof(int2)));
  DCUDA(cudaMemcpy(b->d_descs, descs.data(), descs.size() * sizeof(ClassDesc), cudaMemcpyHostToDevice));
  DCUDA(cudaMemcpy(b->d_work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice));
  b->nwork = (long long)work.size();
  b->ndesc = (int)descs.size();
  b->smem = smem;
  b->grid = b->tiers.empty() ? 0 : b->tiers[0].grid;
  // capture the whole batched build in one graph
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  cudaStream_t cap;
  DCUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  DCUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  b->graph_kernels = 0;
  for (int m = 0; m < nmol; ++m) {
    lx3c_dfj* p = b->mols[m];
    cudaMemsetAsync(p->d_gacc, 0, p->naux_ao * kFixBytes, cap);
    cudaMemsetAsync(p->d_Jacc, 0, p->nao * p->nao * kFixBytes, cap);
    for (auto& g : p->groups) {
      launch_pair_precompute(p->orb->dev(), g.d_pairs, (long long)g.counts.size(), g.Ka, g.Kb, g.d_pairrec,
                             g.d_pairab, cap);
      launch_aux_precompute(p->aux->dev(), g.d_auxs, (long long)g.auxs.size(), g.Kc, g.d_auxrec, g.d_auxc, cap);
      b->graph_kernels += 2;
    }
  }
  for (size_t t = 0; t < b->tiers.size(); ++t) {
    const auto& T = b->tiers[t];
    cudaMemsetAsync(b->d_counter + t, 0, sizeof(unsigned long long), cap);
    launch_persistent(b->d_descs, b->d_work + T.off, T.n, b->d_counter + t, T.grid, T.smem, T.three, cap);
    b->graph_kernels += 1;
  }
  for (int m = 0; m < nmol; ++m) {
    launch_fix_finish(b->mols[m]->d_gacc, b->mols[m]->naux_ao, gamma[m], cap);
    launch_fix_finish_J(b->mols[m]->d_Jacc, b->mols[m]->nao, J[m], cap);
    b->graph_kernels += 2;
  }
  cudaError_t ce = cudaStreamEndCapture(cap, &b->graph);
  if (ce != cudaSuccess) {
    cudaStreamDestroy(cap);
    return dfail(LX3C_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  }
  ce = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (ce == cudaSuccess) ce = capture_branches(b, descs, grids, order, cap);
  cudaStreamDestroy(cap);
  if (ce != cudaSuccess) return dfail(LX3C_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  (void)stream;
  return LX3C_OK;
}

lx3c_status lx3c_batch_execute(lx3c_batch* b, int mode, void* stream) {
  if (!b) return dfail(LX3C_EINVAL, "null batch");
  if (b->D.empty()) return dfail(LX3C_EINVAL, "batch not bound (lx3c_batch_bind)");
  cudaStream_t st = (cudaStream_t)stream;
  if (mode == 1 || mode == 2) {
    DCUDA(cudaGraphLaunch(mode == 1 ? b->exec : b->exec2, st));
    return LX3C_OK;
  }
  if (mode != 0) return dfail(LX3C_EINVAL, "mode must be 0, 1 or 2");
  for (size_t m = 0; m < b->mols.size(); ++m) {
    lx3c_status rc = lx3c_dfj_execute(b->mols[m], b->D[m], b->c[m], b->gamma[m], b->J[m], stream);
    if (rc) return rc;
  }
  return LX3C_OK;
}

lx3c_status lx3c_batch_info(const lx3c_batch* b, double* out, int n) {
  if (!b || (!out && n > 0)) return dfail(LX3C_EINVAL, "null pointer");
  double tasks = 0, nint = 0, flops = 0, slots = 0;
  for (auto* p : b->mols)
    for (auto& g : p->groups) {
      tasks += (double)g.ntasks; nint += g.nint; flops += g.flops;
      for (auto& L : g.L) slots += (double)L.ntiles * L.desc.T;
    }
  const double v[] = {(double)b->mols.size(), tasks, nint, flops, (double)b->plain_launches,
                      (double)b->graph_kernels, (double)b->nwork, (double)b->ndesc, (double)b->smem,
                      (double)b->grid, (double)b->tuned.size(), (double)b->ntuned_measured,
                      (double)b->branch_kernels, (double)kBranches, slots, (double)b->tiers.size()};
  for (int i = 0; i < n && i < 16; ++i) out[i] = v[i];
  return LX3C_OK;
}

}  // extern "C"
