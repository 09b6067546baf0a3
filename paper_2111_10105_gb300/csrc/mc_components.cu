// Connected components of the mesh graph and the anchor-coverage check of
// the decoder (Section III, Eq. 12).
//
// L 1 = 0 holds row by row (Eq. 3), so every connected component's indicator
// vector lies in the null space of L, and L^T L + P^T P of Eq. 12 is
// singular unless each component holds at least one anchor.  The handle
// labels every vertex with the smallest vertex index of its component once
// per connectivity; a decode then checks the stream's anchor set against the
// labels before any solve work is enqueued.
//
// Labelling: a lock-free union-find.  One thread per vertex walks its
// neighbours j > i and links the two roots, always the larger root under the
// smaller one with a compare-and-swap, so no cycle can form and each final
// root is the smallest vertex of its component; path halving shortens the
// chains as they are walked.  A second pass writes every vertex's root.
#include <algorithm>

#include "mc_internal.cuh"

namespace mc {
namespace {

__device__ __forceinline__ int cc_find(volatile int32_t* parent, int x) {
  // path halving: parent[x] <- parent[parent[x]] along the walk; concurrent
  // walkers only ever replace a parent by one of its ancestors
  while (true) {
    const int p = parent[x];
    if (p == x) return x;
    const int gp = parent[p];
    if (gp != p) parent[x] = gp;
    x = gp;
  }
}

__global__ void k_cc_init(int n, int32_t* __restrict__ parent) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    parent[i] = i;
}

__global__ void k_cc_hook(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                          int n, int32_t* parent) {
  volatile int32_t* vp = parent;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e1 = row_ptr[i + 1];
    for (int e = row_ptr[i]; e < e1; ++e) {
      const int j = col_idx[e];
      if (j <= i) continue;              // every undirected edge once
      int a = cc_find(vp, i), b = cc_find(vp, j);
      while (a != b) {
        if (a < b) { const int t = a; a = b; b = t; }   // link the larger root a under b
        const int old = atomicCAS(&parent[a], a, b);
        if (old == a) break;
        a = cc_find(vp, old);            // a was linked meanwhile: continue from its root
        b = cc_find(vp, b);
      }
    }
  }
}

__global__ void k_cc_flatten(int n, int32_t* parent, int32_t* __restrict__ comp) {
  volatile int32_t* vp = parent;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    comp[i] = cc_find(vp, i);
}

// flag[comp[a]] = 1 for every anchor a in range (indices outside [0, n) are
// left to the bitstream checks)
__global__ void k_cover_mark(const int32_t* __restrict__ comp, int n,
                             const int32_t* __restrict__ anchors, int n_c,
                             uint8_t* __restrict__ flag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_c; i += gridDim.x * blockDim.x) {
    const int a = anchors[i];
    if (a >= 0 && a < n) flag[comp[a]] = 1;
  }
}

__global__ void k_cover_check(const int32_t* __restrict__ comp, int n,
                              const uint8_t* __restrict__ flag, uint32_t* status) {
  bool bad = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    bad |= comp[i] == i && flag[i] == 0;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NO_ANCHOR);
}

int grid_for(long long count) {
  return (int)std::max<long long>(1, std::min<long long>((count + 255) / 256, 152 * 16));
}

}  // namespace

void component_labels(const int32_t* row_ptr, const int32_t* col_idx, int n, int32_t* parent,
                      int32_t* comp, cudaStream_t s, Launches& L) {
  const int g = grid_for(n);
  k_cc_init<<<g, 256, 0, s>>>(n, parent);
  k_cc_hook<<<g, 256, 0, s>>>(row_ptr, col_idx, n, parent);
  k_cc_flatten<<<g, 256, 0, s>>>(n, parent, comp);
  L.add(3);
}

void anchor_coverage(const int32_t* comp, int n, const int32_t* anchors, int n_c, uint8_t* flag,
                     uint32_t* status, cudaStream_t s, Launches& L) {
  cudaMemsetAsync(flag, 0, (size_t)n, s);
  if (n_c > 0) {
    k_cover_mark<<<grid_for(n_c), 256, 0, s>>>(comp, n, anchors, n_c, flag);
    L.add(1);
  }
  k_cover_check<<<grid_for(n), 256, 0, s>>>(comp, n, flag, status);
  L.add(1);
}

}  // namespace mc
