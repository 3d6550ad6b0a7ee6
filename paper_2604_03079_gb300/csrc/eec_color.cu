// Jones-Plassmann colouring on the GPU (the parallel colouring the paper cites for its conflict
// graph, Sec. I).
//
// A device is coloured once every conflicting device of higher priority is coloured, and it
// takes the smallest colour none of those uses. With priority = position in a visiting order
// this is exactly the sequential greedy colouring of Sec. I / Sec. II in that order (each device
// sees the same set of already-coloured neighbours), so the result is bit-exact with the host
// greedy. Ready devices are processed in rounds from a worklist; a device counts its pending
// higher-priority neighbours and joins the next worklist when the count reaches zero. Edges are
// implicit: two devices conflict when they share a conflict node (node -> device lists).
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "eec_internal.h"

namespace eec {

namespace {

struct JP {
  const int* node_ptr;
  const int* node_dev;
  const int* dev_ptr;
  const int* dev_node;
  const uint32_t* prio;
  int* col;
  int* cnt;
};

__global__ void k_jp_init(JP g, int N, int* wl, int* wl_size) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  const uint32_t pv = g.prio[v];
  int c = 0;
  for (int p = g.dev_ptr[v]; p < g.dev_ptr[v + 1]; ++p) {
    const int node = g.dev_node[p];
    for (int q = g.node_ptr[node]; q < g.node_ptr[node + 1]; ++q) {
      const int w = g.node_dev[q];
      if (w != v && g.prio[w] > pv) ++c;
    }
  }
  g.cnt[v] = c;
  g.col[v] = -1;
  if (c == 0) wl[atomicAdd(wl_size, 1)] = v;
}

__global__ void k_jp_round(JP g, const int* wl, int n_wl, int* next, int* next_size) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_wl) return;
  const int v = wl[i];
  const uint32_t pv = g.prio[v];
  const int d0 = g.dev_ptr[v], d1 = g.dev_ptr[v + 1];
  // smallest colour unused by higher-priority neighbours, 64 candidates per pass
  int base = 0;
  for (;;) {
    unsigned long long used = 0ull;
    for (int p = d0; p < d1; ++p) {
      const int node = g.dev_node[p];
      for (int q = g.node_ptr[node]; q < g.node_ptr[node + 1]; ++q) {
        const int w = g.node_dev[q];
        if (w == v || g.prio[w] < pv) continue;
        const int cw = g.col[w] - base;
        if (cw >= 0 && cw < 64) used |= 1ull << cw;
      }
    }
    if (used != ~0ull) {
      base += __ffsll((long long)~used) - 1;
      break;
    }
    base += 64;
  }
  g.col[v] = base;
  for (int p = d0; p < d1; ++p) {
    const int node = g.dev_node[p];
    for (int q = g.node_ptr[node]; q < g.node_ptr[node + 1]; ++q) {
      const int w = g.node_dev[q];
      if (w != v && g.prio[w] < pv && atomicSub(g.cnt + w, 1) == 1)
        next[atomicAdd(next_size, 1)] = w;
    }
  }
}

template <class T>
cudaError_t up(T** p, const std::vector<T>& h) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (h.empty() ? 1 : h.size()) * sizeof(T));
  if (e != cudaSuccess || h.empty()) return e;
  return cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

int jp_color(int N, const std::vector<int>& node_ptr, const std::vector<int>& node_dev,
             const std::vector<int>& dev_ptr, const std::vector<int>& dev_node,
             const std::vector<uint32_t>& prio, std::vector<int>& col, int* n_colors,
             std::string& err) {
  col.assign(N, 0);
  *n_colors = 0;
  if (N == 0) return EEC_OK;
  JP g{};
  int *wl0 = nullptr, *wl1 = nullptr, *sizes = nullptr;
  int *np = nullptr, *nd = nullptr, *dp = nullptr, *dnn = nullptr;
  uint32_t* pr = nullptr;
  int rc = EEC_OK;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess && x != cudaSuccess) e = x; };
  chk(up(&np, node_ptr));
  chk(up(&nd, node_dev));
  chk(up(&dp, dev_ptr));
  chk(up(&dnn, dev_node));
  chk(up(&pr, prio));
  chk(cudaMalloc(&g.col, sizeof(int) * N));
  chk(cudaMalloc(&g.cnt, sizeof(int) * N));
  chk(cudaMalloc(&wl0, sizeof(int) * N));
  chk(cudaMalloc(&wl1, sizeof(int) * N));
  chk(cudaMalloc(&sizes, sizeof(int) * 2));
  if (e == cudaSuccess) {
    g.node_ptr = np; g.node_dev = nd; g.dev_ptr = dp; g.dev_node = dnn; g.prio = pr;
    chk(cudaMemset(sizes, 0, sizeof(int) * 2));
    k_jp_init<<<(N + 255) / 256, 256>>>(g, N, wl0, sizes);
    chk(cudaGetLastError());
    int n_wl = 0, done = 0;
    chk(cudaMemcpy(&n_wl, sizes, sizeof(int), cudaMemcpyDeviceToHost));
    while (e == cudaSuccess && n_wl > 0) {
      done += n_wl;
      chk(cudaMemset(sizes + 1, 0, sizeof(int)));
      k_jp_round<<<(n_wl + 127) / 128, 128>>>(g, wl0, n_wl, wl1, sizes + 1);
      chk(cudaGetLastError());
      chk(cudaMemcpy(&n_wl, sizes + 1, sizeof(int), cudaMemcpyDeviceToHost));
      std::swap(wl0, wl1);
      if (done > N) break;
    }
    if (e == cudaSuccess && done != N) {
      rc = EEC_EINVAL;
      err = "Jones-Plassmann left devices uncoloured (priorities not unique?)";
    }
    if (e == cudaSuccess) chk(cudaMemcpy(col.data(), g.col, sizeof(int) * N, cudaMemcpyDeviceToHost));
  }
  if (e != cudaSuccess) {
    rc = EEC_ECUDA;
    err = std::string("Jones-Plassmann: ") + cudaGetErrorString(e);
  }
  cudaFree(np); cudaFree(nd); cudaFree(dp); cudaFree(dnn); cudaFree(pr);
  cudaFree(g.col); cudaFree(g.cnt); cudaFree(wl0); cudaFree(wl1); cudaFree(sizes);
  int C = 0;
  for (int v : col) C = v + 1 > C ? v + 1 : C;
  *n_colors = C;
  return rc;
}

}  // namespace eec
