// Tile-callback form of the DF-J build (lx3c_dfj_execute_tiles): the
// paper's end-user DF-J interface (Sec. 3) receives tiles of the density
// matrix and writes tiles of J through callables, so that the library makes
// no assumption about how or where the caller stores them (any layout, any
// distribution over processes).  Here the callables are C function pointers
// with a user pointer; every tile is a rectangle of whole shells.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/lx3c.h"
#include "lx3c_internal.h"

namespace lx3c {
const lx3c_basis* dfj_orbital_basis(const lx3c_dfj* plan);
}

using namespace lx3c;

namespace {

lx3c_status tfail(lx3c_status s, const std::string& m) {
  set_last_error("dfj_execute_tiles: " + m);
  return s;
}

// D[i][j] = D[j][i] for i > j (the caller supplies the upper triangle of tiles)
__global__ void mirror_upper(double* __restrict__ D, long long n) {
  const long long i = blockIdx.y * (long long)blockDim.y + threadIdx.y;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n && j < i) D[i * n + j] = D[j * n + i];
}

struct TileBuffers {
  double *D = nullptr, *J = nullptr, *c = nullptr, *g = nullptr, *stage = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ~TileBuffers() {
    cudaFree(D); cudaFree(J); cudaFree(c); cudaFree(g);
    if (stage) cudaFreeHost(stage);
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
  }
};

}  // namespace

extern "C" lx3c_status lx3c_dfj_execute_tiles(lx3c_dfj* plan, int64_t tile_ao, lx3c_tile_get_fn get_D,
                                              lx3c_tile_put_fn put_J, void* user, const double* c, double* gamma,
                                              void* stream) {
  if (!plan || !get_D || !c || (!put_J && !gamma)) return tfail(LX3C_EINVAL, "null pointer");
  if (tile_ao < 1) return tfail(LX3C_EINVAL, "tile_ao must be >= 1");
  double info[7];
  lx3c_status rc = lx3c_dfj_info(plan, info, 7);
  if (rc) return rc;
  const long long nao = (long long)info[5], naux = (long long)info[6];
  const lx3c_basis* orb = dfj_orbital_basis(plan);
  // shell-aligned block edges of about tile_ao AOs (a shell never splits)
  std::vector<long long> edge{0};
  long long ao = 0;
  for (int64_t s = 0; s < orb->nshell; ++s) {
    ao += 2 * orb->l[s] + 1;
    if (ao - edge.back() >= tile_ao || s + 1 == orb->nshell) edge.push_back(ao);
  }
  const int nb = (int)edge.size() - 1;
  long long maxb = 0;
  for (int b = 0; b < nb; ++b) maxb = std::max(maxb, edge[b + 1] - edge[b]);
  cudaStream_t st = (cudaStream_t)stream;
  TileBuffers tb;
  const size_t stage1 = (size_t)maxb * maxb;
  if (cudaMalloc(&tb.D, (size_t)nao * nao * 8) != cudaSuccess || cudaMalloc(&tb.J, (size_t)nao * nao * 8) != cudaSuccess ||
      cudaMalloc(&tb.c, naux * 8) != cudaSuccess || cudaMalloc(&tb.g, naux * 8) != cudaSuccess ||
      cudaMallocHost(&tb.stage, 2 * stage1 * 8) != cudaSuccess)
    return tfail(LX3C_ENOMEM, "device or page-locked buffer allocation failed");
  for (auto& e : tb.ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return tfail(LX3C_ECUDA, "event");
  // D: upper triangle of tiles through the callable, two staging buffers in turn
  int buf = 0;
  bool used[2] = {false, false};
  for (int bi = 0; bi < nb; ++bi)
    for (int bj = bi; bj < nb; ++bj) {
      const long long r0 = edge[bi], nr = edge[bi + 1] - r0, c0 = edge[bj], nc = edge[bj + 1] - c0;
      double* hs = tb.stage + buf * stage1;
      if (used[buf] && cudaEventSynchronize(tb.ev[buf]) != cudaSuccess) return tfail(LX3C_ECUDA, "event wait");
      if (get_D(user, r0, nr, c0, nc, hs, nc) != 0) {
        cudaStreamSynchronize(st);
        return tfail(LX3C_EINVAL, "get_D callable reported an error");
      }
      if (cudaMemcpy2DAsync(tb.D + r0 * nao + c0, nao * 8, hs, nc * 8, nc * 8, nr, cudaMemcpyHostToDevice, st) !=
              cudaSuccess ||
          cudaEventRecord(tb.ev[buf], st) != cudaSuccess)
        return tfail(LX3C_ECUDA, "tile copy to the device");
      used[buf] = true;
      buf ^= 1;
    }
  dim3 blk(32, 8), grd((unsigned)((nao + 31) / 32), (unsigned)((nao + 7) / 8));
  mirror_upper<<<grd, blk, 0, st>>>(tb.D, nao);
  if (cudaGetLastError() != cudaSuccess) return tfail(LX3C_ECUDA, "mirror launch");
  if (cudaMemcpyAsync(tb.c, c, naux * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return tfail(LX3C_ECUDA, "c copy");
  rc = lx3c_dfj_execute(plan, tb.D, tb.c, tb.g, put_J ? tb.J : nullptr, stream);
  if (rc) return rc;
  if (gamma && cudaMemcpyAsync(gamma, tb.g, naux * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return tfail(LX3C_ECUDA, "gamma copy");
  if (cudaStreamSynchronize(st) != cudaSuccess) return tfail(LX3C_ECUDA, "build");
  if (!put_J) return LX3C_OK;
  // J: every tile, the copy of the next tile in flight while the caller takes the current one
  std::vector<std::pair<int, int>> order;
  for (int bi = 0; bi < nb; ++bi)
    for (int bj = 0; bj < nb; ++bj) order.push_back({bi, bj});
  auto issue = [&](size_t k, int b) {
    const long long r0 = edge[order[k].first], nr = edge[order[k].first + 1] - r0;
    const long long c0 = edge[order[k].second], nc = edge[order[k].second + 1] - c0;
    cudaError_t e = cudaMemcpy2DAsync(tb.stage + b * stage1, nc * 8, tb.J + r0 * nao + c0, nao * 8, nc * 8, nr,
                                      cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(tb.ev[b], st);
    return e;
  };
  if (issue(0, 0) != cudaSuccess) return tfail(LX3C_ECUDA, "tile copy to the host");
  for (size_t k = 0; k < order.size(); ++k) {
    const int b = (int)(k & 1);
    if (k + 1 < order.size() && issue(k + 1, b ^ 1) != cudaSuccess) return tfail(LX3C_ECUDA, "tile copy to the host");
    if (cudaEventSynchronize(tb.ev[b]) != cudaSuccess) return tfail(LX3C_ECUDA, "event wait");
    const long long r0 = edge[order[k].first], nr = edge[order[k].first + 1] - r0;
    const long long c0 = edge[order[k].second], nc = edge[order[k].second + 1] - c0;
    if (put_J(user, r0, nr, c0, nc, tb.stage + b * stage1, nc) != 0) {
      cudaStreamSynchronize(st);
      return tfail(LX3C_EINVAL, "put_J callable reported an error");
    }
  }
  return LX3C_OK;
}
