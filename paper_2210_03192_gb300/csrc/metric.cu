// Density-fitting metric and solve (the step between gamma and J in a DF-J
// build, Sec. 1 and Sec. 4 of arXiv:2210.03192: the fitted density is
// c = V^{-1} gamma with V_PQ = (P|Q) over the auxiliary basis):
//   lx3c_metric_plan/execute  V_PQ = (P|Q) by the class kernel, as the
//                              3-centre integral (P 1|Q) whose bra partner is
//                              the constant function 1 (an s Gaussian with
//                              exponent 0), stored straight into V
//   lx3c_cholesky             blocked right-looking Cholesky V = L L^T in FP64
//   lx3c_cholesky_solve       L L^T X = B by blocked forward and backward
//                              substitution
//   lx3c_dfj_coulomb          gamma -> c = V^{-1} gamma -> J in one call
//
// Cholesky kernels (row-major, lower triangle; the strictly upper triangle is
// never written):
//   chol_diag    one CTA factors the nb x nb diagonal block in shared memory
//   chol_trsm    rows below it: L21 = A21 L11^{-T}, one thread per row
//   chol_update  A22 -= L21 L21^T on 128 x 128 tiles of the lower triangle,
//                8 x 8 FMA accumulators per thread (the FP64 pipe, not shared
//                memory or HBM, bounds this GEMM on GB300)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/lx3c.h"
#include "lx3c_internal.h"

namespace lx3c {
cudaError_t launch_pair_precompute(const DevBasis& orb, const int32_t* pairs, long long npair, int Ka, int Kb,
                                   double* rec, double* ab, cudaStream_t st, int scale_a = 0, int scale_b = 0);
cudaError_t launch_aux_precompute(const DevBasis& aux, const int32_t* auxs, long long naux, int Kc, double* rec,
                                  double* cxyz, cudaStream_t st);
cudaError_t launch_eri3c(const ClassDesc& d, int grid, cudaStream_t st);
int eri3c_occupancy(int smem_bytes);
}  // namespace lx3c

using namespace lx3c;

namespace {

lx3c_status mfail(lx3c_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

#define MCUDA(expr)                                                                                         \
  do {                                                                                                      \
    cudaError_t e_ = (expr);                                                                                \
    if (e_ != cudaSuccess) return mfail(LX3C_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));   \
  } while (0)

constexpr int kNB = 64;        // panel width of the Cholesky and the solves
constexpr int kTile = 128;     // trailing-update tile
constexpr int kLd = kTile + 1; // padded shared-memory row of the update operands
constexpr int kTrsmRows = 128; // rows per CTA of the panel solve

// ---------------------------------------------------------------------------
// Cholesky
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) chol_diag(double* __restrict__ A, long long lda, long long k, int nb,
                                                 int* __restrict__ info, const double* __restrict__ diag0,
                                                 double drop_tol) {
  __shared__ double s[kNB][kNB + 1];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nb * nb; idx += 256) {
    const int i = idx / nb, j = idx - i * nb;
    s[i][j] = j <= i ? A[(k + i) * lda + k + j] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      double dj = s[j][j];
      if (diag0) {
        // drop mode: a pivot at or below drop_tol of the original diagonal
        // marks a function dependent on the earlier ones; an infinite pivot
        // zeroes its column below and its coefficient in the solves
        if (!(dj > drop_tol * diag0[k + j])) {
          if (info) ++*info;
          s[j][j] = __longlong_as_double(0x7FF0000000000000LL);
        } else {
          s[j][j] = sqrt(dj);
        }
      } else {
        if (!(dj > 0.0)) {  // not positive definite: record the first such pivot, carry NaN on
          if (info && *info == 0) *info = (int)(k + j + 1);
          dj = nan("");
        }
        s[j][j] = sqrt(dj);
      }
    }
    __syncthreads();
    const double piv = s[j][j];
    for (int i = j + 1 + tid; i < nb; i += 256) s[i][j] /= piv;
    __syncthreads();
    const int m = nb - j - 1;
    for (int idx = tid; idx < m * m; idx += 256) {
      const int r = idx / m, c = idx - r * m;
      if (c <= r) s[j + 1 + r][j + 1 + c] = fma(-s[j + 1 + r][j], s[j + 1 + c][j], s[j + 1 + r][j + 1 + c]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nb * nb; idx += 256) {
    const int i = idx / nb, j = idx - i * nb;
    if (j <= i) A[(k + i) * lda + k + j] = s[i][j];
  }
}

// Rows r0 .. r0+kTrsmRows-1 (r0 = k + nb + blockIdx.x * kTrsmRows) of the
// panel: x L11^T = a, i.e. forward substitution with L11 per row.
__global__ void __launch_bounds__(kTrsmRows) chol_trsm(double* __restrict__ A, long long lda, long long k, int nb,
                                                       long long n) {
  extern __shared__ double sm[];
  double* L = sm;                     // [kNB][kNB + 1]
  double* X = sm + kNB * (kNB + 1);   // [kTrsmRows][kNB + 1]
  const int tid = threadIdx.x;
  const long long r0 = k + nb + (long long)blockIdx.x * kTrsmRows;
  for (int idx = tid; idx < nb * nb; idx += kTrsmRows) {
    const int i = idx / nb, j = idx - i * nb;
    L[i * (kNB + 1) + j] = j <= i ? A[(k + i) * lda + k + j] : 0.0;
  }
  for (int idx = tid; idx < kTrsmRows * nb; idx += kTrsmRows) {
    const int r = idx / nb, j = idx - r * nb;
    X[r * (kNB + 1) + j] = r0 + r < n ? A[(r0 + r) * lda + k + j] : 0.0;
  }
  __syncthreads();
  double* x = X + tid * (kNB + 1);
  for (int j = 0; j < nb; ++j) {
    double v = x[j];
    for (int p = 0; p < j; ++p) v = fma(-x[p], L[j * (kNB + 1) + p], v);
    x[j] = v / L[j * (kNB + 1) + j];
  }
  __syncthreads();
  for (int idx = tid; idx < kTrsmRows * nb; idx += kTrsmRows) {
    const int r = idx / nb, j = idx - r * nb;
    if (r0 + r < n) A[(r0 + r) * lda + k + j] = X[r * (kNB + 1) + j];
  }
}

// Lower tile (bi, bj), bj <= bi, of the trailing matrix (rows/cols from
// r0 = k + nb): A[i][j] -= sum_p L[i][k+p] L[j][k+p] for j <= i.
__global__ void __launch_bounds__(256) chol_update(double* __restrict__ A, long long lda, long long k, int nb,
                                                   long long n) {
  extern __shared__ double sm[];
  double* As = sm;              // [nb][kLd]: rows of tile bi, transposed
  double* Bs = sm + nb * kLd;   // [nb][kLd]: rows of tile bj, transposed
  const long long x = blockIdx.x;
  long long bi = (long long)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
  while (bi * (bi + 1) / 2 > x) --bi;
  while ((bi + 1) * (bi + 2) / 2 <= x) ++bi;
  const long long bj = x - bi * (bi + 1) / 2;
  const long long r0 = k + nb, ri = r0 + bi * kTile, rj = r0 + bj * kTile;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kTile * nb; idx += 256) {
    const int r = idx / nb, p = idx - r * nb;
    As[p * kLd + r] = ri + r < n ? A[(ri + r) * lda + k + p] : 0.0;
    Bs[p * kLd + r] = rj + r < n ? A[(rj + r) * lda + k + p] : 0.0;
  }
  __syncthreads();
  const int ty = tid >> 4, tx = tid & 15;
  double acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.0;
  for (int p = 0; p < nb; ++p) {
    double a[8], b[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = As[p * kLd + ty + 16 * r];
#pragma unroll
    for (int c = 0; c < 8; ++c) b[c] = Bs[p * kLd + tx + 16 * c];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const long long i = ri + ty + 16 * r;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const long long j = rj + tx + 16 * c;
      if (j <= i) A[i * lda + j] -= acc[r][c];
    }
  }
}

// ---------------------------------------------------------------------------
// triangular solves, B row-major [n][nrhs]
// ---------------------------------------------------------------------------

// B[k..k+nb) <- L_kk^{-1} B[k..k+nb) (forward) or L_kk^{-T} (backward).
__global__ void __launch_bounds__(256) solve_diag(const double* __restrict__ L, long long lda, long long k, int nb,
                                                  double* __restrict__ B, long long nrhs, int backward) {
  __shared__ double s[kNB][kNB + 1];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nb * nb; idx += 256) {
    const int i = idx / nb, j = idx - i * nb;
    s[i][j] = j <= i ? L[(k + i) * lda + k + j] : 0.0;
  }
  __syncthreads();
  for (long long q = tid; q < nrhs; q += 256) {
    double* b = B + k * nrhs + q;
    if (!backward) {
      for (int j = 0; j < nb; ++j) {
        double v = b[j * nrhs];
        for (int p = 0; p < j; ++p) v = fma(-s[j][p], b[p * nrhs], v);
        b[j * nrhs] = v / s[j][j];
      }
    } else {
      for (int j = nb - 1; j >= 0; --j) {
        double v = b[j * nrhs];
        for (int p = j + 1; p < nb; ++p) v = fma(-s[p][j], b[p * nrhs], v);
        b[j * nrhs] = v / s[j][j];
      }
    }
  }
}

// Forward update: rows i >= k + nb, B[i] -= L[i][k..k+nb) B[k..k+nb); one
// warp per row, lanes over the panel columns, shuffle reduction per rhs.
__global__ void __launch_bounds__(256) solve_update_fwd(const double* __restrict__ L, long long lda, long long k,
                                                        int nb, double* __restrict__ B, long long nrhs, long long n) {
  const int lane = threadIdx.x & 31;
  const long long i = k + nb + (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= n) return;
  const double l0 = lane < nb ? L[i * lda + k + lane] : 0.0;
  const double l1 = lane + 32 < nb ? L[i * lda + k + lane + 32] : 0.0;
  for (long long q = 0; q < nrhs; ++q) {
    double v = 0.0;
    if (lane < nb) v = l0 * B[(k + lane) * nrhs + q];
    if (lane + 32 < nb) v = fma(l1, B[(k + lane + 32) * nrhs + q], v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) B[i * nrhs + q] -= v;
  }
}

// Backward update: rows j < k, B[j] -= sum_i L[k+i][j] B[k+i]; one thread per
// (row j, rhs q), reading a column of the block row (coalesced across j).
__global__ void __launch_bounds__(256) solve_update_bwd(const double* __restrict__ L, long long lda, long long k,
                                                        int nb, double* __restrict__ B, long long nrhs) {
  const long long w = (long long)blockIdx.x * 256 + threadIdx.x;
  if (w >= k * nrhs) return;
  const long long j = w / nrhs, q = w - j * nrhs;
  double v = 0.0;
  for (int i = 0; i < nb; ++i) v = fma(L[(k + i) * lda + j], B[(k + i) * nrhs + q], v);
  B[j * nrhs + q] -= v;
}

bool g_attr_done = false;

cudaError_t chol_attributes() {
  if (g_attr_done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(chol_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(2 * kNB * kLd * sizeof(double)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chol_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((kNB + kTrsmRows) * (kNB + 1) * sizeof(double)));
  if (e == cudaSuccess) g_attr_done = true;
  return e;
}

__global__ void copy_diag(const double* __restrict__ A, long long lda, long long n, double* __restrict__ d) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) d[i] = A[i * lda + i];
}

cudaError_t cholesky_launches(double* A, long long n, long long lda, int* info, const double* diag0,
                              double drop_tol, cudaStream_t st) {
  cudaError_t e = chol_attributes();
  for (long long k = 0; k < n && e == cudaSuccess; k += kNB) {
    const int nb = (int)std::min<long long>(kNB, n - k);
    chol_diag<<<1, 256, 0, st>>>(A, lda, k, nb, info, diag0, drop_tol);
    e = cudaGetLastError();
    const long long m = n - k - nb;
    if (m <= 0 || e != cudaSuccess) continue;
    chol_trsm<<<(unsigned)((m + kTrsmRows - 1) / kTrsmRows), kTrsmRows,
                (kNB + kTrsmRows) * (kNB + 1) * sizeof(double), st>>>(A, lda, k, nb, n);
    e = cudaGetLastError();
    if (e != cudaSuccess) continue;
    const long long T = (m + kTile - 1) / kTile;
    chol_update<<<(unsigned)(T * (T + 1) / 2), 256, 2 * nb * kLd * sizeof(double), st>>>(A, lda, k, nb, n);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t solve_launches(const double* L, long long n, long long lda, double* B, long long nrhs, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (long long k = 0; k < n && e == cudaSuccess; k += kNB) {
    const int nb = (int)std::min<long long>(kNB, n - k);
    solve_diag<<<1, 256, 0, st>>>(L, lda, k, nb, B, nrhs, 0);
    e = cudaGetLastError();
    const long long m = n - k - nb;
    if (m > 0 && e == cudaSuccess) {
      solve_update_fwd<<<(unsigned)((m + 7) / 8), 256, 0, st>>>(L, lda, k, nb, B, nrhs, n);
      e = cudaGetLastError();
    }
  }
  const long long last = ((n - 1) / kNB) * kNB;
  for (long long k = last; k >= 0 && e == cudaSuccess; k -= kNB) {
    const int nb = (int)std::min<long long>(kNB, n - k);
    solve_diag<<<1, 256, 0, st>>>(L, lda, k, nb, B, nrhs, 1);
    e = cudaGetLastError();
    if (k > 0 && e == cudaSuccess) {
      solve_update_bwd<<<(unsigned)((k * nrhs + 255) / 256), 256, 0, st>>>(L, lda, k, nb, B, nrhs);
      e = cudaGetLastError();
    }
  }
  return e;
}

}  // namespace

// ---------------------------------------------------------------------------
// metric plan
// ---------------------------------------------------------------------------

struct lx3c_metric {
  const lx3c_basis* aux = nullptr;
  lx3c_basis* bra = nullptr;  // the aux shells followed by the unit s shell (exponent 0)
  long long naux_ao = 0;
  struct Group {
    int l = 0, K = 0;
    std::vector<int> shells;
    int32_t* d_pairs = nullptr;   // (shell, unit shell)
    int32_t* d_kets = nullptr;
    int4* d_sub = nullptr;
    int* d_prim = nullptr;
    int4* d_pair_ao = nullptr;
    int* d_aux_ao = nullptr;
    double* d_pairrec = nullptr;
    double* d_pairab = nullptr;
    double* d_auxrec = nullptr;
    double* d_auxc = nullptr;
  };
  std::vector<Group> groups;
  struct Launch {
    ClassDesc desc;
    int grid = 1;
  };
  std::vector<Launch> launches;
  double flops = 0;
};

extern "C" {

void lx3c_metric_destroy(lx3c_metric* p) {
  if (!p) return;
  for (auto& g : p->groups) {
    cudaFree(g.d_pairs); cudaFree(g.d_kets); cudaFree(g.d_sub); cudaFree(g.d_prim); cudaFree(g.d_pair_ao);
    cudaFree(g.d_aux_ao); cudaFree(g.d_pairrec); cudaFree(g.d_pairab); cudaFree(g.d_auxrec); cudaFree(g.d_auxc);
  }
  lx3c_basis_destroy(p->bra);
  delete p;
}

lx3c_status lx3c_metric_plan(lx3c_metric** out, const lx3c_basis* aux, void* stream) {
  if (!out) return mfail(LX3C_EINVAL, "metric_plan: null output pointer");
  *out = nullptr;
  if (!aux || aux->nshell <= 0) return mfail(LX3C_EINVAL, "metric_plan: empty aux basis");
  for (int64_t s = 0; s < aux->nshell; ++s)
    if (aux->l[s] > LX3C_LMAX_AUX) return mfail(LX3C_ENOTSUP, "metric_plan: aux shell beyond the supported l");
  DevState* ds;
  int rc = device_state_get(&ds);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  std::unique_ptr<lx3c_metric, void (*)(lx3c_metric*)> p(new lx3c_metric, lx3c_metric_destroy);
  p->aux = aux;
  // bra basis: every aux shell, then the constant function 1 = exp(-0 r^2)
  lx3c_basis* b = new lx3c_basis;
  p->bra = b;
  b->nshell = aux->nshell + 1;
  b->nprim = aux->nprim + 1;
  b->l = aux->l; b->l.push_back(0);
  b->k = aux->k; b->k.push_back(1);
  b->atom = aux->atom; b->atom.push_back(-1);
  b->off = aux->off; b->off.push_back(aux->nprim);
  b->xyz = aux->xyz; b->xyz.insert(b->xyz.end(), {0.0, 0.0, 0.0});
  b->exps = aux->exps; b->exps.push_back(0.0);
  b->coefs = aux->coefs; b->coefs.push_back(1.0);
  rc = basis_upload(b, st);
  if (rc) return rc;
  const int unit = (int)aux->nshell;
  std::vector<int> aq(aux->nshell + 1, 0);
  for (int64_t s = 0; s < aux->nshell; ++s) aq[s + 1] = aq[s] + 2 * aux->l[s] + 1;
  p->naux_ao = aq[aux->nshell];
  std::map<std::pair<int, int>, std::vector<int>> byclass;
  for (int64_t s = 0; s < aux->nshell; ++s) byclass[{aux->l[s], aux->k[s]}].push_back((int)s);
  for (auto& kv : byclass) {
    lx3c_metric::Group g;
    g.l = kv.first.first;
    g.K = kv.first.second;
    g.shells = kv.second;
    const long long ns = (long long)g.shells.size();
    std::vector<int32_t> pairs(2 * ns);
    std::vector<int4> sub(ns), pao(ns);
    std::vector<int> prim(ns * g.K), aao(ns);
    for (long long i = 0; i < ns; ++i) {
      pairs[2 * i] = g.shells[i];
      pairs[2 * i + 1] = unit;
      sub[i] = int4{(int)i, (int)(i * g.K), g.K, 0};
      for (int r = 0; r < g.K; ++r) prim[i * g.K + r] = r;
      pao[i] = int4{aq[g.shells[i]], 0, 0, 0};
      aao[i] = aq[g.shells[i]];
    }
    MCUDA(cudaMalloc(&g.d_pairs, ns * 8));
    MCUDA(cudaMalloc(&g.d_kets, ns * 4));
    MCUDA(cudaMalloc(&g.d_sub, ns * sizeof(int4)));
    MCUDA(cudaMalloc(&g.d_prim, prim.size() * 4));
    MCUDA(cudaMalloc(&g.d_pair_ao, ns * sizeof(int4)));
    MCUDA(cudaMalloc(&g.d_aux_ao, ns * 4));
    MCUDA(cudaMalloc(&g.d_pairrec, (size_t)ns * g.K * kPairRec * 8));
    MCUDA(cudaMalloc(&g.d_pairab, (size_t)ns * 3 * 8));
    MCUDA(cudaMalloc(&g.d_auxrec, (size_t)ns * g.K * kAuxRec * 8));
    MCUDA(cudaMalloc(&g.d_auxc, (size_t)ns * 3 * 8));
    MCUDA(cudaMemcpyAsync(g.d_pairs, pairs.data(), ns * 8, cudaMemcpyHostToDevice, st));
    MCUDA(cudaMemcpyAsync(g.d_kets, g.shells.data(), ns * 4, cudaMemcpyHostToDevice, st));
    MCUDA(cudaMemcpyAsync(g.d_sub, sub.data(), ns * sizeof(int4), cudaMemcpyHostToDevice, st));
    MCUDA(cudaMemcpyAsync(g.d_prim, prim.data(), prim.size() * 4, cudaMemcpyHostToDevice, st));
    MCUDA(cudaMemcpyAsync(g.d_pair_ao, pao.data(), ns * sizeof(int4), cudaMemcpyHostToDevice, st));
    MCUDA(cudaMemcpyAsync(g.d_aux_ao, aao.data(), ns * 4, cudaMemcpyHostToDevice, st));
    p->groups.push_back(g);
  }
  // one class launch (lP 0 | lQ) per pair of groups
  for (auto& gp : p->groups)
    for (auto& gq : p->groups) {
      const ClassTables* ct;
      try {
        ct = &class_tables(gp.l, 0, gq.l, 1);
      } catch (std::exception& e) {
        return mfail(LX3C_ENOTSUP, std::string("metric_plan: ") + e.what());
      }
      DevClass* dc;
      rc = device_class_get(ds, *ct, &dc);
      if (rc) return rc;
      lx3c_metric::Launch L;
      ClassDesc& d = L.desc;
      const long long np = (long long)gp.shells.size(), nq = (long long)gq.shells.size();
      if (fill_class_desc(d, *ct, *dc, ds, 0, gp.K, gp.K, gq.K, nq) < 0)
        return mfail(LX3C_ENOTSUP, "metric_plan: class does not fit in shared memory");
      d.npair = np;
      d.naux = nq;
      d.nsub = np;
      d.ntile_aux = (int)((nq + d.T - 1) / d.T);
      d.ntiles = np * d.ntile_aux;
      d.subpairs = gp.d_sub;
      d.primidx = gp.d_prim;
      d.pairrec = gp.d_pairrec; d.pairab = gp.d_pairab;
      d.auxrec = gq.d_auxrec; d.auxc = gq.d_auxc;
      d.digest = 3;
      d.ldD = p->naux_ao;
      d.pair_ao = gp.d_pair_ao;
      d.aux_ao = gq.d_aux_ao;
      const int occ = eri3c_occupancy(d.smem_doubles * 8);
      L.grid = (int)std::min<long long>(d.ntiles, (long long)dev_nsm(ds) * occ * 8);
      double fl = 0;
      lx3c_class_flops(gp.l, 0, gq.l, gp.K, gq.K, 1, &fl);
      p->flops += fl * (double)np * (double)nq;
      p->launches.push_back(L);
    }
  MCUDA(cudaStreamSynchronize(st));
  *out = p.release();
  return LX3C_OK;
}

lx3c_status lx3c_metric_execute(lx3c_metric* p, double* V, void* stream) {
  if (!p || !V) return mfail(LX3C_EINVAL, "metric_execute: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  for (auto& g : p->groups) {
    const long long ns = (long long)g.shells.size();
    MCUDA(launch_pair_precompute(p->bra->dev(), g.d_pairs, ns, g.K, 1, g.d_pairrec, g.d_pairab, st));
    MCUDA(launch_aux_precompute(p->aux->dev(), g.d_kets, ns, g.K, g.d_auxrec, g.d_auxc, st));
  }
  for (auto& L : p->launches) {
    ClassDesc d = L.desc;
    d.out = V;
    MCUDA(launch_eri3c(d, L.grid, st));
  }
  return LX3C_OK;
}

lx3c_status lx3c_metric_info(const lx3c_metric* p, double* out, int n) {
  if (!p || (!out && n > 0)) return mfail(LX3C_EINVAL, "metric_info: null pointer");
  const double v[] = {(double)p->naux_ao, (double)p->groups.size(), (double)p->launches.size(),
                      2.0 * p->groups.size() + p->launches.size(), p->flops,
                      (double)p->aux->nshell * (double)p->aux->nshell};
  for (int i = 0; i < n && i < 6; ++i) out[i] = v[i];
  return LX3C_OK;
}

lx3c_status lx3c_cholesky(double* A, int64_t n, int64_t lda, double drop_tol, int32_t* info, void* stream) {
  if (!A || n < 1 || lda < n) return mfail(LX3C_EINVAL, "cholesky: null matrix, n < 1 or lda < n");
  if (!(drop_tol >= 0.0 && drop_tol < 1.0)) return mfail(LX3C_EINVAL, "cholesky: drop_tol must be in [0, 1)");
  cudaStream_t st = (cudaStream_t)stream;
  if (info) MCUDA(cudaMemsetAsync(info, 0, sizeof(int32_t), st));
  double* diag0 = nullptr;
  if (drop_tol > 0.0) {
    MCUDA(cudaMallocAsync(&diag0, (size_t)n * sizeof(double), st));
    copy_diag<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(A, lda, n, diag0);
    MCUDA(cudaGetLastError());
  }
  cudaError_t e = cholesky_launches(A, n, lda, info, diag0, drop_tol, st);
  if (diag0) cudaFreeAsync(diag0, st);
  MCUDA(e);
  return LX3C_OK;
}

lx3c_status lx3c_cholesky_solve(const double* L, int64_t n, int64_t lda, double* B, int64_t nrhs, void* stream) {
  if (!L || !B || n < 1 || lda < n || nrhs < 1) return mfail(LX3C_EINVAL, "cholesky_solve: bad argument");
  MCUDA(solve_launches(L, n, lda, B, nrhs, (cudaStream_t)stream));
  return LX3C_OK;
}

lx3c_status lx3c_dfj_coulomb(lx3c_dfj* plan, const double* L, int64_t lda, const double* D, double* gamma,
                             double* c, double* J, void* stream) {
  if (!plan || !L || !D || !gamma || !c || !J) return mfail(LX3C_EINVAL, "dfj_coulomb: null pointer");
  double info[7];
  lx3c_status rc = lx3c_dfj_info(plan, info, 7);
  if (rc) return rc;
  const long long naux_ao = (long long)info[6];
  if (lda < naux_ao) return mfail(LX3C_EINVAL, "dfj_coulomb: lda smaller than the aux AO count");
  cudaStream_t st = (cudaStream_t)stream;
  rc = lx3c_dfj_execute(plan, D, c, gamma, nullptr, stream);  // gamma only; c is not read
  if (rc) return rc;
  MCUDA(cudaMemcpyAsync(c, gamma, naux_ao * sizeof(double), cudaMemcpyDeviceToDevice, st));
  MCUDA(solve_launches(L, naux_ao, lda, c, 1, st));
  return lx3c_dfj_execute(plan, D, c, nullptr, J, stream);
}

}  // extern "C"
