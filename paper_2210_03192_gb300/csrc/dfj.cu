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
// in digest mode: gamma and J are accumulated with FP64 atomics from each
// tile's block in shared memory; a final kernel symmetrises J.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lx3c.h"
#include "lx3c_internal.h"

namespace lx3c {
cudaError_t launch_pair_precompute(const DevBasis& orb, const int32_t* pairs, long long npair, int Ka, int Kb,
                                   double* rec, double* ab, cudaStream_t st);
cudaError_t launch_aux_precompute(const DevBasis& aux, const int32_t* auxs, long long naux, int Kc, double* rec,
                                  double* cxyz, cudaStream_t st);
cudaError_t launch_eri3c(const ClassDesc& d, int grid, cudaStream_t st);
int eri3c_occupancy(int smem_bytes);
}  // namespace lx3c

using namespace lx3c;

namespace {

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

constexpr double kPi = 3.14159265358979323846;

// sqrt of a Schwarz-type estimate of max |(ab|ab)| for a shell pair: the
// (ss|ss) value of each primitive pair times the rms size of (x-A)^la (x-B)^lb
// under the product Gaussian.
double q_pair(const lx3c_basis* b, int sa, int sb) {
  const double* A = &b->xyz[3 * sa];
  const double* B = &b->xyz[3 * sb];
  double ab2 = 0;
  for (int x = 0; x < 3; ++x) ab2 += (A[x] - B[x]) * (A[x] - B[x]);
  double q = 0;
  for (int ia = 0; ia < b->k[sa]; ++ia)
    for (int ib = 0; ib < b->k[sb]; ++ib) {
      const double za = b->exps[b->off[sa] + ia], zb = b->exps[b->off[sb] + ib], g = za + zb;
      double pa2 = 0, pb2 = 0;
      for (int x = 0; x < 3; ++x) {
        const double P = (za * A[x] + zb * B[x]) / g;
        pa2 += (P - A[x]) * (P - A[x]);
        pb2 += (P - B[x]) * (P - B[x]);
      }
      q += std::fabs(b->coefs[b->off[sa] + ia] * b->coefs[b->off[sb] + ib]) * std::exp(-za * zb / g * ab2) *
           std::sqrt(2.0 * std::pow(kPi, 2.5) / (g * g * std::sqrt(2.0 * g))) *
           std::pow(pa2 + 0.5 / g, 0.5 * b->l[sa]) * std::pow(pb2 + 0.5 / g, 0.5 * b->l[sb]);
    }
  return q;
}

double q_aux(const lx3c_basis* b, int s) {
  double q = 0;
  for (int i = 0; i < b->k[s]; ++i) {
    const double z = b->exps[b->off[s] + i];
    q += std::fabs(b->coefs[b->off[s] + i]) * std::sqrt(2.0 * std::pow(kPi, 2.5) / (z * z * std::sqrt(2.0 * z))) *
         std::pow(0.5 / z, 0.5 * b->l[s]);
  }
  return q;
}

struct DfjLaunch {
  ClassDesc desc;
  int grid = 1;
  long long ntiles = 0;
  int4* d_sub = nullptr;
  int* d_prim = nullptr;
  int4* d_tiles = nullptr;
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
};

}  // namespace

struct lx3c_dfj {
  const lx3c_basis* orb = nullptr;
  const lx3c_basis* aux = nullptr;
  long long nao = 0, naux_ao = 0;
  double tol = 0;
  std::vector<DfjGroup> groups;
};

extern "C" {

void lx3c_dfj_destroy(lx3c_dfj* p) {
  if (!p) return;
  for (auto& g : p->groups) {
    cudaFree(g.d_pairs); cudaFree(g.d_auxs); cudaFree(g.d_pair_ao); cudaFree(g.d_aux_ao);
    cudaFree(g.d_pairrec); cudaFree(g.d_pairab); cudaFree(g.d_auxrec); cudaFree(g.d_auxc);
    for (auto& L : g.L) {
      cudaFree(L.d_sub); cudaFree(L.d_prim); cudaFree(L.d_tiles);
    }
  }
  delete p;
}

lx3c_status lx3c_dfj_plan(lx3c_dfj** out, const lx3c_basis* orb, const lx3c_basis* aux, double schwarz_tol,
                          void* stream) {
  if (!out) return dfail(LX3C_EINVAL, "null output pointer");
  *out = nullptr;
  if (!orb || !aux) return dfail(LX3C_EINVAL, "null basis");
  if (orb->nshell <= 0 || aux->nshell <= 0) return dfail(LX3C_EINVAL, "empty basis");
  if (!(schwarz_tol >= 0.0)) return dfail(LX3C_EINVAL, "negative or NaN tolerance");
  for (int64_t s = 0; s < orb->nshell; ++s)
    if (orb->l[s] > LX3C_LMAX_ORB) return dfail(LX3C_ENOTSUP, "orbital shell beyond the supported l");
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
        const double thr = ql[i] > 0 ? schwarz_tol / ql[i] : 1e308;
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
  // per group: orientation split, tiles, device lists
  for (auto& g : p->groups) {
    const long long np = (long long)g.counts.size(), na = (long long)g.auxs.size();
    const int nbra = (2 * g.la + 1) * (2 * g.lb + 1), nket = 2 * g.lc + 1;
    double fl = 0;
    if (lx3c_class_flops(g.la, g.lb, g.lc, g.Ka * g.Kb, g.Kc, 1, &fl)) return LX3C_ENOTSUP;
    g.flops = (fl + 4.0 * nbra * nket) * (double)g.ntasks;
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
      if (fill_class_desc(d, *ct, *dc, ds, o, kmax[o], Kab, g.Kc, cmax) < 0)
        return dfail(LX3C_ENOTSUP, "class does not fit in shared memory");
      std::vector<int4> tiles;
      for (size_t s = 0; s < sub[o].size(); ++s) {
        const int cnt = g.counts[sub[o][s].x];
        for (int a0 = 0; a0 < cnt; a0 += d.T) tiles.push_back(int4{(int)s, a0, std::min(d.T, cnt - a0), 0});
      }
      L.ntiles = (long long)tiles.size();
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
      d.ldD = p->nao;
      d.pair_ao = g.d_pair_ao;
      d.aux_ao = g.d_aux_ao;
      const int occ = eri3c_occupancy(d.smem_doubles * 8);
      L.grid = (int)std::min<long long>(L.ntiles, (long long)dev_nsm(ds) * occ * 8);
    }
  }
  DCUDA(cudaStreamSynchronize(st));
  *out = p.release();
  return LX3C_OK;
}

lx3c_status lx3c_dfj_execute(lx3c_dfj* p, const double* D, const double* c, double* gamma, double* J, void* stream) {
  if (!p) return dfail(LX3C_EINVAL, "null plan");
  if (!D || !c || !gamma || !J) return dfail(LX3C_EINVAL, "null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  DCUDA(cudaMemsetAsync(gamma, 0, p->naux_ao * 8, st));
  DCUDA(cudaMemsetAsync(J, 0, p->nao * p->nao * 8, st));
  for (auto& g : p->groups) {
    const long long np = (long long)g.counts.size(), na = (long long)g.auxs.size();
    DCUDA(launch_pair_precompute(p->orb->dev(), g.d_pairs, np, g.Ka, g.Kb, g.d_pairrec, g.d_pairab, st));
    DCUDA(launch_aux_precompute(p->aux->dev(), g.d_auxs, na, g.Kc, g.d_auxrec, g.d_auxc, st));
    for (auto& L : g.L) {
      if (!L.ntiles) continue;
      ClassDesc d = L.desc;
      d.D = D;
      d.cvec = c;
      d.gamma = gamma;
      d.J = J;
      DCUDA(launch_eri3c(d, L.grid, st));
    }
  }
  dim3 blk(32, 8), grd((unsigned)((p->nao + 31) / 32), (unsigned)((p->nao + 7) / 8));
  symmetrize<<<grd, blk, 0, st>>>(J, p->nao);
  DCUDA(cudaGetLastError());
  return LX3C_OK;
}

lx3c_status lx3c_dfj_info(const lx3c_dfj* p, double* out, int n) {
  if (!p || (!out && n > 0)) return dfail(LX3C_EINVAL, "null pointer");
  double tasks = 0, nint = 0, flops = 0, launches = 1;
  for (auto& g : p->groups) {
    tasks += (double)g.ntasks;
    nint += g.nint;
    flops += g.flops;
    launches += 2 + (g.L[0].ntiles > 0) + (g.L[1].ntiles > 0);
  }
  const double v[] = {(double)p->groups.size(), tasks, nint, flops, launches, (double)p->nao, (double)p->naux_ao};
  for (int i = 0; i < n && i < 7; ++i) out[i] = v[i];
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
