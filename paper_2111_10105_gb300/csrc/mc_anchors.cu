// Anchor selection by farthest points (Section III-B: n_c anchors, "uniformly
// distributed" over the mesh, against the seeded random choice the codec
// makes by default; the paper leaves the best choice open in Section V).
//
// Greedy farthest-point selection (Gonzalez's k-center heuristic) in
// Euclidean distance over one pose: start from a given vertex, then add, n_c
// - 1 times, the vertex whose squared distance to its nearest chosen vertex
// is largest (equal distances: the lowest index).  Squared distances are
// formed with separately rounded operations, (dx*dx + dy*dy) + dz*dz, so the
// choice does not depend on contraction into fused multiply-adds.
//
// One launch per added vertex: every CTA lowers its vertices' distances with
// the previous choice and proposes its farthest vertex; the last CTA to finish
// (an atomic ticket, no waiting) takes the farthest proposal, marks it chosen
// (distance -1, never chosen again) and resets the ticket.  A final one-CTA
// pass writes the chosen set in ascending index order.
#include <algorithm>
#include <math.h>

#include "mc_internal.cuh"

namespace mc {
namespace {

constexpr int kFpsThreads = 256;

struct Far {
  double d;
  int i;
};

// the farther of two proposals; equal distances keep the lower index
__device__ __forceinline__ Far farther(Far a, Far b) {
  if (b.d > a.d || (b.d == a.d && b.i < a.i)) return b;
  return a;
}

__device__ __forceinline__ double dist2(const double* __restrict__ xyz, int i, int a) {
  const double dx = __dsub_rn(xyz[3LL * i], xyz[3LL * a]);
  const double dy = __dsub_rn(xyz[3LL * i + 1], xyz[3LL * a + 1]);
  const double dz = __dsub_rn(xyz[3LL * i + 2], xyz[3LL * a + 2]);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ Far block_farthest(Far f, Far* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Far g;
    g.d = __shfl_down_sync(0xffffffffu, f.d, o);
    g.i = __shfl_down_sync(0xffffffffu, f.i, o);
    f = farther(f, g);
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = f;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < kFpsThreads / 32; ++w) f = farther(f, sh[w]);
  return f;   // valid in thread 0
}

__global__ void k_fps_init(int n, int start, double* mind, int32_t* chosen, uint32_t* ticket) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    mind[i] = i == start ? -1.0 : INFINITY;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    chosen[0] = start;
    *ticket = 0;
  }
}

// choose chosen[t] from the distances to chosen[0..t-1]
__global__ void __launch_bounds__(kFpsThreads) k_fps_step(int n, const double* __restrict__ xyz,
                                                          double* mind, int32_t* chosen, int t,
                                                          Far* part, uint32_t* ticket) {
  __shared__ Far sh[kFpsThreads / 32];
  __shared__ bool last_cta;
  const int prev = chosen[t - 1];
  Far f{-2.0, 0x7fffffff};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double m = mind[i];
    if (m >= 0.0) {   // chosen vertices keep -1
      m = fmin(m, dist2(xyz, i, prev));
      mind[i] = m;
    }
    f = farther(f, Far{m, i});
  }
  f = block_farthest(f, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = f;
    __threadfence();
    last_cta = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last_cta) return;
  __threadfence();
  Far g{-2.0, 0x7fffffff};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const volatile Far* vp = part + b;
    g = farther(g, Far{vp->d, vp->i});
  }
  __syncthreads();   // sh is reused
  g = block_farthest(g, sh);
  if (threadIdx.x == 0) {
    chosen[t] = g.i;
    mind[g.i] = -1.0;
    *ticket = 0;
  }
}

// the chosen vertices (distance -1) in ascending order, one CTA
__global__ void __launch_bounds__(1024) k_fps_compact(int n, const double* __restrict__ mind,
                                                      int32_t* __restrict__ out) {
  __shared__ int warp_count[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < n; c0 += 1024) {
    const int i = c0 + threadIdx.x;
    const bool sel = i < n && mind[i] < 0.0;
    const unsigned m = __ballot_sync(0xffffffffu, sel);
    if (lane == 0) warp_count[warp] = __popc(m);
    __syncthreads();
    int off = base;
    for (int w = 0; w < warp; ++w) off += warp_count[w];
    if (sel) out[off + __popc(m & ((1u << lane) - 1u))] = i;
    __syncthreads();
    if (threadIdx.x == 0)
      for (int w = 0; w < 32; ++w) base += warp_count[w];
    __syncthreads();
  }
}

}  // namespace
}  // namespace mc

using namespace mc;

mesh_codec_status_t mesh_codec_farthest_anchors(int n, int n_c, const double* xyz, int start,
                                                int32_t* anchors, void* stream) {
  if (n < 1 || n_c < 1 || n_c > n || start < 0 || start >= n || !xyz || !anchors)
    return MC_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (int)std::min<long long>((n + kFpsThreads - 1) / kFpsThreads, 152 * 4);
  const size_t bytes = sizeof(double) * (size_t)n + sizeof(Far) * blocks +
                       sizeof(int32_t) * (size_t)n_c + 64;
  char* ws = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&ws), bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return MC_E_OOM;
  }
  double* mind = reinterpret_cast<double*>(ws);
  Far* part = reinterpret_cast<Far*>(ws + sizeof(double) * (size_t)n);
  int32_t* chosen = reinterpret_cast<int32_t*>(part + blocks);
  uint32_t* ticket = reinterpret_cast<uint32_t*>(chosen + n_c);
  k_fps_init<<<blocks, kFpsThreads, 0, s>>>(n, start, mind, chosen, ticket);
  for (int t = 1; t < n_c; ++t)
    k_fps_step<<<blocks, kFpsThreads, 0, s>>>(n, xyz, mind, chosen, t, part, ticket);
  k_fps_compact<<<1, 1024, 0, s>>>(n, mind, anchors);
  const cudaError_t e = cudaGetLastError();
  cudaFreeAsync(ws, s);
  return e == cudaSuccess ? MC_OK : MC_E_CUDA;
}
