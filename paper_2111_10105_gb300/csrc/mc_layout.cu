// Layout transforms between the caller's frame-major positions [F][n][3]
// (the sequence A = [M_1; ...; M_F] of Section II) and the codec's
// vertex-major [n][3F] matrix (column c*F + f = coordinate c of frame f).
// Both are 32 x 32 (frames x vertices) shared-memory tile transposes; every
// global access is a contiguous run of >= 256 bytes.
#include <algorithm>

#include "mc_internal.cuh"

namespace mc {

static constexpr int kT = 32;

__global__ void __launch_bounds__(256) k_frames_to_vm(const double* __restrict__ pos,
                                                      double* __restrict__ X, int F, int n) {
  __shared__ double tile[kT][3 * kT + 1];  // [frame][vertex*3 + c]
  const int f0 = blockIdx.y * kT, i0 = blockIdx.x * kT;
  const int W = 3 * F;
  // load: for each frame row, 96 consecutive doubles (32 vertices x 3)
  for (int e = threadIdx.x; e < kT * 3 * kT; e += blockDim.x) {
    int fr = e / (3 * kT), q = e % (3 * kT);
    int f = f0 + fr, i = i0 + q / 3;
    if (f < F && i < n) tile[fr][q] = pos[((long long)f * n + i) * 3 + (q % 3)];
  }
  __syncthreads();
  // store: for each (vertex, coordinate), 32 consecutive frames
  for (int e = threadIdx.x; e < kT * 3 * kT; e += blockDim.x) {
    int fr = e % kT, vc = e / kT;  // vc = vertex*3 + c
    int v = vc / 3, c = vc % 3;
    int f = f0 + fr, i = i0 + v;
    if (f < F && i < n) X[(long long)i * W + c * F + f] = tile[fr][v * 3 + c];
  }
}

__global__ void __launch_bounds__(256) k_vm_to_frames(const double* __restrict__ X,
                                                      double* __restrict__ pos, int F, int n) {
  __shared__ double tile[kT][3 * kT + 1];
  const int f0 = blockIdx.y * kT, i0 = blockIdx.x * kT;
  const int W = 3 * F;
  for (int e = threadIdx.x; e < kT * 3 * kT; e += blockDim.x) {
    int fr = e % kT, vc = e / kT;
    int v = vc / 3, c = vc % 3;
    int f = f0 + fr, i = i0 + v;
    if (f < F && i < n) tile[fr][v * 3 + c] = X[(long long)i * W + c * F + f];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kT * 3 * kT; e += blockDim.x) {
    int fr = e / (3 * kT), q = e % (3 * kT);
    int f = f0 + fr, i = i0 + q / 3;
    if (f < F && i < n) pos[((long long)f * n + i) * 3 + (q % 3)] = tile[fr][q];
  }
}

void frames_to_vertex_major(const double* pos, double* X, int F, int n, cudaStream_t s,
                            Launches& L) {
  dim3 grid((n + kT - 1) / kT, (F + kT - 1) / kT);
  k_frames_to_vm<<<grid, 256, 0, s>>>(pos, X, F, n);
  L.add(1);
}

void vertex_major_to_frames(const double* X, double* pos, int F, int n, cudaStream_t s,
                            Launches& L) {
  dim3 grid((n + kT - 1) / kT, (F + kT - 1) / kT);
  k_vm_to_frames<<<grid, 256, 0, s>>>(X, pos, F, n);
  L.add(1);
}

}  // namespace mc
