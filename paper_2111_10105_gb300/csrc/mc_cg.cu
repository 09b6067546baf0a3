// Decoder solve (Eq. 12): the anchored least-squares problem
//   min_X ||L X - delta~||^2 + ||P X - a^||^2
// through its normal equations (L^T L + P^T P) X = L^T delta~ + P^T a^, solved
// for all W columns at once by Jacobi-preconditioned conjugate gradients with
// an independent step length per column (the paper's parallel
// reconstruction, Section IV (v)).  The operator is applied as two Laplacian
// sweeps, never assembled.
//
// Each iteration is six kernels over the [n][W] vectors:
//   1. T = L P                          (SpMM over the adjacency)
//   2. Q = L^T T + P^T P P, pAp partial (SpMM + dot, per row block)
//   3. alpha = rz / pAp                 (per column, fixed-order reduction)
//   4. X += alpha P, R -= alpha Q, partial rz = R.(D^-1 R), rr = R.R
//   5. beta, convergence, active count  (per column, fixed-order reduction)
//   6. P = D^-1 R + beta P
// Dot products are reduced deterministically: per (row block, column)
// partials in a fixed order, then one CTA per column with a fixed reduction
// tree.  A converged column is frozen (alpha = beta = 0, no more updates),
// so its result does not depend on the other columns.
#include <algorithm>
#include <math.h>

#include "mc_internal.cuh"

namespace mc {

static constexpr int kCgThreads = 256;  // 32 columns x 8 row lanes

CgGeom cg_geometry_rows(int n, int W, int rpb) {
  CgGeom g{};
  g.n = n;
  g.W = W;
  rpb = std::max(8, (rpb + 7) / 8 * 8);
  g.rows_per_block = rpb;
  g.row_blocks = (n + rpb - 1) / rpb;
  return g;
}

// Default shape: about 16 CTAs of 32 columns x 8 row lanes per SM, and at
// most kMaxRows rows per CTA.  CTAs are dispatched in blockIdx order with
// the column block fastest, so short row blocks keep every resident CTA on
// one narrow band of rows: the neighbour rows a gather re-reads (the band's
// width plus the adjacency's bandwidth, times the row length) then stay in
// L2, where long row blocks spread the resident CTAs over the whole matrix
// and evict them (measured on the 99,856-vertex grid with 1,192 FP32
// columns: 3x the algorithmic DRAM reads with 1,561-row blocks).  Measured
// per FP32 iteration with 192 columns: 32 rows 0.286 ms, 64 rows 0.241 ms,
// 128 rows 0.229 ms, 256 rows 0.253 ms (99,856-vertex grid); 128 rows 0.605
// ms against 0.640 ms at 256 on the 262,144-vertex grid.
static constexpr int kMaxRows = 128;

CgGeom cg_geometry(int n, int W) {
  int col_tiles = (W + 31) / 32;
  long long target = std::max(1, (152 * 16) / std::max(1, col_tiles));
  const int rows = (int)std::min<long long>(kMaxRows, (n + target - 1) / target);
  return cg_geometry_rows(n, W, rows);
}

// the autotuner's candidates: the default rows per CTA times 1/2, 1, 2, 4
static const int kTuneNum[4] = {1, 1, 2, 4}, kTuneDen[4] = {2, 1, 1, 1};

size_t cg_partials_elems(int n, int W) {
  const CgGeom g = cg_geometry(n, W);
  const CgGeom h = cg_geometry_rows(n, W, g.rows_per_block / 2);   // most row blocks
  return (size_t)std::max(g.row_blocks, h.row_blocks) * W * 2;
}

// Combine the 8 row-lane partial sums of a column in fixed order and store
// the CTA's partial for (row block, column).
__device__ __forceinline__ void cta_col_partial(double v, double* sh, double* out, int col,
                                                int W, bool valid) {
  const int lane = threadIdx.x & 31, rl = threadIdx.x >> 5;
  sh[rl * 32 + lane] = v;
  __syncthreads();
  if (rl == 0 && valid) {
    double s = sh[lane];
#pragma unroll
    for (int r = 1; r < 8; ++r) s += sh[r * 32 + lane];
    out[(long long)blockIdx.y * W + col] = s;
  }
  __syncthreads();
}

// Vector kernels, templated on the vector type T: double (FP64 mode) or
// float (mixed modes: FP32 vectors and operator).  Dot products of FP32
// vectors are accumulated per thread by Dot2 (Ogita, Rump, Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 2005: TwoProduct by FMA and
// TwoSum, all on the FP32 pipe), which is as accurate as accumulating in
// twice the working precision, and the per-thread results are combined in
// FP64.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);            // a*b = p + e exactly
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));  // s+p = t+err
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <typename T>
__global__ void __launch_bounds__(kCgThreads) k_cg_init(CgGeom g, const double* __restrict__ B,
                                                        T* __restrict__ X, T* __restrict__ R,
                                                        T* __restrict__ P,
                                                        const T* __restrict__ inv_diag,
                                                        double* __restrict__ partials) {
  __shared__ double sh[256];
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rl = threadIdx.x >> 5;
  const bool valid = col < g.W;
  const long long r0 = (long long)blockIdx.y * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  DotAcc<T> rz, bb;
  if (valid) {
    for (long long i = r0 + rl; i < r1; i += 8) {
      long long e = i * g.W + col;
      const T b = (T)B[e];
      const T z = b * inv_diag[i];
      X[e] = (T)0;
      R[e] = b;
      P[e] = z;
      rz.add(b, z);
      bb.add(b, b);
    }
  }
  const long long plane = (long long)g.row_blocks * g.W;
  cta_col_partial(rz.value(), sh, partials, col, g.W, valid);
  cta_col_partial(bb.value(), sh, partials + plane, col, g.W, valid);
}

// One CTA (256 threads) per column: fixed-order sum of the row-block partials
// (a strided sum per thread, a shuffle tree per warp, then the 8 warps in
// order); the result is valid in thread 0.  A whole CTA per column keeps
// many loads in flight where one warp per column was latency-bound.
__device__ __forceinline__ double col_sum(const double* part, int row_blocks, int W, int col) {
  __shared__ double sh[8];
  double s = 0.0;
  for (int b = threadIdx.x; b < row_blocks; b += 256) s += part[(long long)b * W + col];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __syncthreads();   // thread 0 has read the previous call's sums
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < 8; ++w) t += sh[w];
  return t;
}

__global__ void k_cg_init_cols(CgGeom g, const double* __restrict__ partials, double* rz,
                               double* bb, int32_t* done, int32_t* iters) {
  const int col = blockIdx.x;   // grid: one CTA per column
  const long long plane = (long long)g.row_blocks * g.W;
  double a = col_sum(partials, g.row_blocks, g.W, col);
  double b = col_sum(partials + plane, g.row_blocks, g.W, col);
  if (threadIdx.x == 0) {
    rz[col] = a;
    bb[col] = b;
    done[col] = (b == 0.0) ? 1 : 0;
    iters[col] = 0;
  }
}

// Neighbour values are loaded four at a time (independent loads in flight)
// and summed in ascending column order, the same order as one at a time.
struct CsrView {
  const int32_t* rp;   // row offsets, indexed by row - r0
  const int32_t* ci;   // column indices
};

// sum over p in [b, e) of V[ci[p]*W + col], ascending p
template <typename T>
__device__ __forceinline__ T gather_sum(const T* __restrict__ V, const int32_t* ci, int b, int e,
                                        int W, int col) {
  T acc = (T)0;
  int p = b;
  for (; p + 4 <= e; p += 4) {
    const int c0 = ci[p], c1 = ci[p + 1], c2 = ci[p + 2], c3 = ci[p + 3];
    const T v0 = V[(long long)c0 * W + col], v1 = V[(long long)c1 * W + col];
    const T v2 = V[(long long)c2 * W + col], v3 = V[(long long)c3 * W + col];
    acc += v0;
    acc += v1;
    acc += v2;
    acc += v3;
  }
  for (; p < e; ++p) acc += V[(long long)ci[p] * W + col];
  return acc;
}

// sum over p in [b, e) of w[ci[p]] * V[ci[p]*W + col] as an FMA chain, ascending p
template <typename T>
__device__ __forceinline__ T gather_wsum(const T* __restrict__ V, const T* __restrict__ w,
                                         const int32_t* ci, int b, int e, int W, int col) {
  T acc = (T)0;
  int p = b;
  for (; p + 4 <= e; p += 4) {
    const int c0 = ci[p], c1 = ci[p + 1], c2 = ci[p + 2], c3 = ci[p + 3];
    const T v0 = V[(long long)c0 * W + col], v1 = V[(long long)c1 * W + col];
    const T v2 = V[(long long)c2 * W + col], v3 = V[(long long)c3 * W + col];
    const T w0 = w[c0], w1 = w[c1], w2 = w[c2], w3 = w[c3];
    acc = fma(w0, v0, acc);
    acc = fma(w1, v1, acc);
    acc = fma(w2, v2, acc);
    acc = fma(w3, v3, acc);
  }
  for (; p < e; ++p) {
    const int c = ci[p];
    acc = fma(w[c], V[(long long)c * W + col], acc);
  }
  return acc;
}

// T = L P for active columns
template <typename T>
__global__ void __launch_bounds__(kCgThreads) k_cg_L(CgGeom g, const int32_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ col_idx,
                                                     const int32_t* __restrict__ deg,
                                                     const T* __restrict__ inv_d, int kind,
                                                     const T* __restrict__ P, T* __restrict__ Tv,
                                                     const int32_t* __restrict__ done) {
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rl = threadIdx.x >> 5;
  const long long r0 = (long long)blockIdx.y * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  const CsrView v{row_ptr + r0, col_idx};
  if (col >= g.W || done[col]) return;
  for (long long i = r0 + rl; i < r1; i += 8) {
    const int b = v.rp[i - r0], e = v.rp[i - r0 + 1];
    const T acc = gather_sum(P, v.ci, b, e, g.W, col);
    const T pi = P[i * g.W + col];
    Tv[i * g.W + col] = (kind == 0) ? fma(-inv_d[i], acc, pi) : fma((T)deg[i], pi, -acc);
  }
}

// Q = L^T T + [anchor] P and partial pAp
template <typename T>
__global__ void __launch_bounds__(kCgThreads) k_cg_LT(CgGeom g, const int32_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col_idx,
                                                      const int32_t* __restrict__ deg,
                                                      const T* __restrict__ inv_d, int kind,
                                                      const uint8_t* __restrict__ is_anchor,
                                                      const T* __restrict__ Tv,
                                                      const T* __restrict__ P, T* __restrict__ Q,
                                                      const int32_t* __restrict__ done,
                                                      double* __restrict__ partials) {
  __shared__ double sh[256];
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rl = threadIdx.x >> 5;
  const long long r0 = (long long)blockIdx.y * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  const CsrView v{row_ptr + r0, col_idx};
  const bool valid = col < g.W && !done[col];
  DotAcc<T> pap;
  if (valid) {
    for (long long j = r0 + rl; j < r1; j += 8) {
      const int b = v.rp[j - r0], e = v.rp[j - r0 + 1];
      const T acc = (kind == 0) ? gather_wsum(Tv, inv_d, v.ci, b, e, g.W, col)
                                : gather_sum(Tv, v.ci, b, e, g.W, col);
      const T tj = Tv[j * g.W + col];
      T q = (kind == 0) ? tj - acc : fma((T)deg[j], tj, -acc);
      const T pj = P[j * g.W + col];
      if (is_anchor[j]) q += pj;
      Q[j * g.W + col] = q;
      pap.add(pj, q);
    }
  }
  cta_col_partial(pap.value(), sh, partials, col, g.W, col < g.W);
}

// alpha = rz / pAp for one column (the whole CTA reduces its partials)
__device__ __forceinline__ void cg_alpha_body(const CgGeom& g, int col,
                                              const double* __restrict__ partials,
                                              const double* __restrict__ rz, double* alpha,
                                              const int32_t* __restrict__ done) {
  double pap = col_sum(partials, g.row_blocks, g.W, col);
  if (threadIdx.x == 0) {
    double a = 0.0;
    if (!done[col] && pap > 0.0) a = rz[col] / pap;
    alpha[col] = a;
  }
}

__global__ void k_cg_alpha(CgGeom g, const double* __restrict__ partials,
                           const double* __restrict__ rz, double* alpha,
                           const int32_t* __restrict__ done, int32_t* active) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *active = 0;
  cg_alpha_body(g, blockIdx.x, partials, rz, alpha, done);   // grid: one CTA per column
}

template <typename T>
__global__ void __launch_bounds__(kCgThreads) k_cg_update(CgGeom g, T* __restrict__ X,
                                                          T* __restrict__ R,
                                                          const T* __restrict__ P,
                                                          const T* __restrict__ Q,
                                                          const T* __restrict__ inv_diag,
                                                          const double* __restrict__ alpha,
                                                          const int32_t* __restrict__ done,
                                                          double* __restrict__ partials) {
  __shared__ double sh[256];
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rl = threadIdx.x >> 5;
  const bool valid = col < g.W && !done[col];
  const long long r0 = (long long)blockIdx.y * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  DotAcc<T> rz, rr;
  if (valid) {
    const T a = (T)alpha[col];
    for (long long i = r0 + rl; i < r1; i += 8) {
      long long e = i * g.W + col;
      X[e] = fma(a, P[e], X[e]);
      T r = fma(-a, Q[e], R[e]);
      R[e] = r;
      T z = r * inv_diag[i];
      rz.add(r, z);
      rr.add(r, r);
    }
  }
  const long long plane = (long long)g.row_blocks * g.W;
  cta_col_partial(rz.value(), sh, partials, col, g.W, col < g.W);
  cta_col_partial(rr.value(), sh, partials + plane, col, g.W, col < g.W);
}

// beta, convergence and the active count for one column
__device__ __forceinline__ void cg_beta_body(const CgGeom& g, int col,
                                             const double* __restrict__ partials, double* rz,
                                             double* rr_out, const double* __restrict__ bb,
                                             double* beta, int32_t* done, int32_t* iters,
                                             double rtol2, int max_iters, int32_t* active) {
  const long long plane = (long long)g.row_blocks * g.W;
  double rzn = col_sum(partials, g.row_blocks, g.W, col);
  double rr = col_sum(partials + plane, g.row_blocks, g.W, col);
  if (threadIdx.x == 0) {
    if (done[col]) {
      beta[col] = 0.0;
      return;
    }
    int it = iters[col] + 1;
    iters[col] = it;
    rr_out[col] = rr;
    if (rr <= rtol2 * bb[col]) {
      done[col] = 1;
      beta[col] = 0.0;
    } else if (it >= max_iters) {
      done[col] = 2;  // cap reached
      beta[col] = 0.0;
    } else {
      beta[col] = rzn / rz[col];
      rz[col] = rzn;
      atomicAdd(active, 1);
    }
  }
}

__global__ void k_cg_beta(CgGeom g, const double* __restrict__ partials, double* rz,
                          double* rr_out, const double* __restrict__ bb, double* beta,
                          int32_t* done, int32_t* iters, double rtol2, int max_iters,
                          int32_t* active) {
  cg_beta_body(g, blockIdx.x, partials, rz, rr_out, bb, beta, done, iters, rtol2, max_iters,
               active);   // grid: one CTA per column
}

// the per-column reductions of a grouped batch (see cg4_grouped_iteration):
// one CTA per column item {solve, column} (CTAs past the table's length return)
__global__ void k_cgg_alpha(const CgSeq* __restrict__ seqs, const int2* __restrict__ cols,
                            const int* __restrict__ n_cols) {
  if ((int)blockIdx.x >= *n_cols) return;
  const int2 w = cols[blockIdx.x];
  const CgSeq& q = seqs[w.x];
  if (w.y == 0 && threadIdx.x == 0) *q.active = 0;
  cg_alpha_body(q.g, w.y, q.partials, q.rz, q.alpha, q.done);
}

__global__ void k_cgg_beta(const CgSeq* __restrict__ seqs, const int2* __restrict__ cols,
                           const int* __restrict__ n_cols) {
  if ((int)blockIdx.x >= *n_cols) return;
  const int2 w = cols[blockIdx.x];
  const CgSeq& q = seqs[w.x];
  cg_beta_body(q.g, w.y, q.partials, q.rz, q.rr, q.bb, q.beta, q.done, q.iters, q.rtol2,
               q.max_iters, q.active);
}

void cgg_alpha(const CgSeq* seqs, const int2* cols, const int* n_cols, int grid, cudaStream_t s) {
  k_cgg_alpha<<<grid, 256, 0, s>>>(seqs, cols, n_cols);
}

void cgg_beta(const CgSeq* seqs, const int2* cols, const int* n_cols, int grid, cudaStream_t s) {
  k_cgg_beta<<<grid, 256, 0, s>>>(seqs, cols, n_cols);
}

template <typename T>
__global__ void __launch_bounds__(kCgThreads) k_cg_dir(CgGeom g, const T* __restrict__ R,
                                                       T* __restrict__ P,
                                                       const T* __restrict__ inv_diag,
                                                       const double* __restrict__ beta,
                                                       const int32_t* __restrict__ done) {
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rl = threadIdx.x >> 5;
  if (col >= g.W || done[col]) return;
  const T b = (T)beta[col];
  const long long r0 = (long long)blockIdx.y * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  for (long long i = r0 + rl; i < r1; i += 8) {
    long long e = i * g.W + col;
    P[e] = fma(b, P[e], R[e] * inv_diag[i]);
  }
}

template <typename T>
static void cg_init_t(const CgGeom& g, const double* B, void* X, void* R, void* P,
                      const void* inv_diag, CgState& st, cudaStream_t s, Launches& L) {
  dim3 grid((g.W + 31) / 32, g.row_blocks);
  k_cg_init<T><<<grid, kCgThreads, 0, s>>>(g, B, (T*)X, (T*)R, (T*)P, (const T*)inv_diag,
                                           st.partials);
  k_cg_init_cols<<<g.W, 256, 0, s>>>(g, st.partials, st.rz, st.bb, st.done, st.iters);
  L.add(2);
}

// CG start from a given X (warm start): R = B - M X with Q = M X already
// computed, P = D^-1 R, rz = R.(D^-1 R), bb = B.B (the stopping rule stays
// relative to ||B||).
template <typename T>
__global__ void __launch_bounds__(kCgThreads) k_cg_init_warm(CgGeom g, const double* __restrict__ B,
                                                             const T* __restrict__ Q,
                                                             T* __restrict__ R, T* __restrict__ P,
                                                             const T* __restrict__ inv_diag,
                                                             double* __restrict__ partials) {
  __shared__ double sh[256];
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rl = threadIdx.x >> 5;
  const bool valid = col < g.W;
  const long long r0 = (long long)blockIdx.y * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  DotAcc<T> rz;
  DotAcc<double> bb;
  if (valid) {
    for (long long i = r0 + rl; i < r1; i += 8) {
      const long long e = i * g.W + col;
      const double b = B[e];
      const T r = (T)(b - (double)Q[e]);
      const T z = r * inv_diag[i];
      R[e] = r;
      P[e] = z;
      rz.add(r, z);
      bb.add(b, b);
    }
  }
  const long long plane = (long long)g.row_blocks * g.W;
  cta_col_partial(rz.value(), sh, partials, col, g.W, valid);
  cta_col_partial(bb.value(), sh, partials + plane, col, g.W, valid);
}

template <typename T>
static void cg_init_warm_t(const CgGeom& g, const int32_t* row_ptr, const int32_t* col_idx,
                           const int32_t* deg, const T* inv_d, const uint8_t* is_anchor, int kind,
                           const double* B, T* X, T* R, T* P, T* Tv, T* Q, const T* inv_diag,
                           CgState& st, cudaStream_t s, Launches& L) {
  dim3 grid((g.W + 31) / 32, g.row_blocks);
  cudaMemsetAsync(st.done, 0, sizeof(int32_t) * g.W, s);
  k_cg_L<T><<<grid, kCgThreads, 0, s>>>(g, row_ptr, col_idx, deg, inv_d, kind, X, Tv, st.done);
  k_cg_LT<T><<<grid, kCgThreads, 0, s>>>(g, row_ptr, col_idx, deg, inv_d, kind, is_anchor, Tv, X,
                                          Q, st.done, st.partials);
  k_cg_init_warm<T><<<grid, kCgThreads, 0, s>>>(g, B, Q, R, P, inv_diag, st.partials);
  k_cg_init_cols<<<g.W, 256, 0, s>>>(g, st.partials, st.rz, st.bb, st.done, st.iters);
  L.add(4);
}

void cg_init_warm(const CgGeom& g, const int32_t* row_ptr, const int32_t* col_idx,
                  const int32_t* deg, const void* inv_d, const uint8_t* is_anchor, int kind,
                  const double* B, void* X, void* R, void* P, void* T, void* Q,
                  const void* inv_diag, CgState& st, int single, cudaStream_t s, Launches& L) {
  if (single)
    cg_init_warm_t<float>(g, row_ptr, col_idx, deg, (const float*)inv_d, is_anchor, kind, B,
                          (float*)X, (float*)R, (float*)P, (float*)T, (float*)Q,
                          (const float*)inv_diag, st, s, L);
  else
    cg_init_warm_t<double>(g, row_ptr, col_idx, deg, (const double*)inv_d, is_anchor, kind, B,
                           (double*)X, (double*)R, (double*)P, (double*)T, (double*)Q,
                           (const double*)inv_diag, st, s, L);
}

void cg_init(const CgGeom& g, const double* B, void* X, void* R, void* P,
             const void* inv_diag, CgState& st, int single, cudaStream_t s, Launches& L) {
  if (cg4_applies(g.W, single)) {
    cg4_init(g, B, (float*)X, (float*)R, (float*)P, (const float*)inv_diag, st.partials, s);
    k_cg_init_cols<<<g.W, 256, 0, s>>>(g, st.partials, st.rz, st.bb, st.done,
                                                 st.iters);
    L.add(2);
  } else if (single) {
    cg_init_t<float>(g, B, X, R, P, inv_diag, st, s, L);
  } else {
    cg_init_t<double>(g, B, X, R, P, inv_diag, st, s, L);
  }
}

// the four-columns-per-thread FP32 iteration (same kernels for alpha / beta)
static void cg_iteration4(const CgGeom& g, const int32_t* row_ptr, const int32_t* col_idx,
                          const int32_t* deg, const float* inv_d, const uint8_t* is_anchor,
                          const float* inv_diag, int kind, float* X, float* R, float* P,
                          float* Tv, float* Q, double rtol, int max_iters, CgState& st,
                          cudaStream_t s, Launches& L, cudaEvent_t* ev) {
  dim3 cgrid(g.W);
  if (ev) cudaEventRecord(ev[0], s);
  cg4_op(g, row_ptr, col_idx, deg, inv_d, kind, is_anchor, P, Tv, Q, st.done, st.partials, s, ev);
  if (ev) cudaEventRecord(ev[2], s);
  k_cg_alpha<<<cgrid, 256, 0, s>>>(g, st.partials, st.rz, st.alpha, st.done, st.active);
  if (ev) cudaEventRecord(ev[3], s);
  cg4_update(g, X, R, P, Q, inv_diag, st.alpha, st.done, st.partials, s);
  if (ev) cudaEventRecord(ev[4], s);
  k_cg_beta<<<cgrid, 256, 0, s>>>(g, st.partials, st.rz, st.rr, st.bb, st.beta, st.done,
                                  st.iters, rtol * rtol, max_iters, st.active);
  if (ev) cudaEventRecord(ev[5], s);
  cg4_dir(g, R, P, inv_diag, st.beta, st.done, s);
  if (ev) cudaEventRecord(ev[6], s);
  L.add(6);
}

template <typename T>
static void cg_iteration_t(const CgGeom& g, const int32_t* row_ptr, const int32_t* col_idx,
                           const int32_t* deg, const T* inv_d, const uint8_t* is_anchor,
                           const T* inv_diag, int kind, T* X, T* R, T* P, T* Tv, T* Q,
                           double rtol, int max_iters, CgState& st, cudaStream_t s, Launches& L,
                           cudaEvent_t* ev) {
  dim3 grid((g.W + 31) / 32, g.row_blocks);
  dim3 cgrid(g.W);
  if (ev) cudaEventRecord(ev[0], s);
  k_cg_L<T><<<grid, kCgThreads, 0, s>>>(g, row_ptr, col_idx, deg, inv_d, kind, P, Tv, st.done);
  if (ev) cudaEventRecord(ev[1], s);
  k_cg_LT<T><<<grid, kCgThreads, 0, s>>>(g, row_ptr, col_idx, deg, inv_d, kind, is_anchor, Tv, P,
                                          Q, st.done, st.partials);
  if (ev) cudaEventRecord(ev[2], s);
  k_cg_alpha<<<cgrid, 256, 0, s>>>(g, st.partials, st.rz, st.alpha, st.done, st.active);
  if (ev) cudaEventRecord(ev[3], s);
  k_cg_update<T><<<grid, kCgThreads, 0, s>>>(g, X, R, P, Q, inv_diag, st.alpha, st.done,
                                              st.partials);
  if (ev) cudaEventRecord(ev[4], s);
  k_cg_beta<<<cgrid, 256, 0, s>>>(g, st.partials, st.rz, st.rr, st.bb, st.beta, st.done,
                                  st.iters, rtol * rtol, max_iters, st.active);
  if (ev) cudaEventRecord(ev[5], s);
  k_cg_dir<T><<<grid, kCgThreads, 0, s>>>(g, R, P, inv_diag, st.beta, st.done);
  if (ev) cudaEventRecord(ev[6], s);
  L.add(6);
}

void cg_iteration(const CgGeom& g, const int32_t* row_ptr, const int32_t* col_idx,
                  const int32_t* deg, const void* inv_d, const uint8_t* is_anchor,
                  const void* inv_diag, int kind, void* X, void* R, void* P, void* T, void* Q,
                  double rtol, int max_iters, CgState& st, int single, cudaStream_t s,
                  Launches& L, cudaEvent_t* ev) {
  if (cg4_applies(g.W, single))
    cg_iteration4(g, row_ptr, col_idx, deg, (const float*)inv_d, is_anchor,
                  (const float*)inv_diag, kind, (float*)X, (float*)R, (float*)P, (float*)T,
                  (float*)Q, rtol, max_iters, st, s, L, ev);
  else if (single)
    cg_iteration_t<float>(g, row_ptr, col_idx, deg, (const float*)inv_d, is_anchor,
                          (const float*)inv_diag, kind, (float*)X,
                          (float*)R, (float*)P, (float*)T, (float*)Q, rtol, max_iters, st, s, L,
                          ev);
  else
    cg_iteration_t<double>(g, row_ptr, col_idx, deg, (const double*)inv_d, is_anchor,
                           (const double*)inv_diag, kind,
                           (double*)X, (double*)R, (double*)P, (double*)T, (double*)Q, rtol,
                           max_iters, st, s, L, ev);
}

// Autotuner of the CG tile shape: times one operator application (k_cg_L +
// k_cg_LT, the two gather kernels) for each candidate rows-per-CTA on the
// current vectors and returns the fastest shape.  The other kernels share it.
CgGeom cg_autotune(int n, int W, const int32_t* row_ptr, const int32_t* col_idx,
                   const int32_t* deg, const void* inv_d, const uint8_t* is_anchor, int kind,
                   void* P, void* T, void* Q, CgState& st, int single, cudaStream_t s,
                   Launches& L) {
  const CgGeom base = cg_geometry(n, W);
  CgGeom best = base;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return base;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return base;
  }
  cudaMemsetAsync(st.done, 0, sizeof(int32_t) * W, s);
  cudaMemsetAsync(P, 0, (single ? 4 : 8) * (size_t)n * W, s);
  for (int c = 0; c < 4; ++c) {
    const CgGeom g = cg_geometry_rows(n, W, base.rows_per_block * kTuneNum[c] / kTuneDen[c]);
    dim3 grid((g.W + 31) / 32, g.row_blocks);
    float ms = 0.f;
    for (int rep = 0; rep < 3; ++rep) {   // first repetition warms up
      cudaEventRecord(e0, s);
      if (cg4_applies(g.W, single)) {
        cg4_op(g, row_ptr, col_idx, deg, (const float*)inv_d, kind, is_anchor, (const float*)P,
               (float*)T, (float*)Q, st.done, st.partials, s, nullptr);
      } else if (single) {
        k_cg_L<float><<<grid, kCgThreads, 0, s>>>(g, row_ptr, col_idx, deg, (const float*)inv_d,
                                                  kind, (const float*)P, (float*)T, st.done);
        k_cg_LT<float><<<grid, kCgThreads, 0, s>>>(g, row_ptr, col_idx, deg, (const float*)inv_d,
                                                   kind, is_anchor, (const float*)T,
                                                   (const float*)P, (float*)Q, st.done,
                                                   st.partials);
      } else {
        k_cg_L<double><<<grid, kCgThreads, 0, s>>>(g, row_ptr, col_idx, deg,
                                                   (const double*)inv_d, kind, (const double*)P,
                                                   (double*)T, st.done);
        k_cg_LT<double><<<grid, kCgThreads, 0, s>>>(g, row_ptr, col_idx, deg,
                                                    (const double*)inv_d, kind, is_anchor,
                                                    (const double*)T, (const double*)P,
                                                    (double*)Q, st.done, st.partials);
      }
      cudaEventRecord(e1, s);
      L.add(2);
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (rep > 0) ms += t;
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = g;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// ------------------------------------------------ iterative refinement (FP64 residuals)
// The refined solve keeps X in FP64 and, per outer step, forms the residual
// R = B - (L^T L + P^T P) X in FP64 (T = L X first), freezes the columns whose
// ||R|| <= rtol ||B||, and lets an FP32 CG solve M D = R for the others.

// R = B - (L^T T + P^T P X) for unfrozen columns (0 for frozen ones), and the
// (row block, column) partials of R.R
__global__ void __launch_bounds__(kCgThreads) k_refine_residual(
    CgGeom g, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
    const int32_t* __restrict__ deg, const double* __restrict__ inv_d, int kind,
    const uint8_t* __restrict__ is_anchor, const double* __restrict__ Tv,
    const double* __restrict__ X, const double* __restrict__ B, double* __restrict__ R,
    const int32_t* __restrict__ frozen, double* __restrict__ partials) {
  __shared__ double sh[256];
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rl = threadIdx.x >> 5;
  const long long r0 = (long long)blockIdx.y * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  const CsrView v{row_ptr + r0, col_idx};
  double rr = 0.0, xx = 0.0;
  if (col < g.W) {
    const bool fz = frozen[col] != 0;
    for (long long j = r0 + rl; j < r1; j += 8) {
      double r = 0.0;
      if (!fz) {
        const int b = v.rp[j - r0], e = v.rp[j - r0 + 1];
        const double acc = (kind == 0) ? gather_wsum(Tv, inv_d, v.ci, b, e, g.W, col)
                                       : gather_sum(Tv, v.ci, b, e, g.W, col);
        const double tj = Tv[j * g.W + col];
        const double xj = X[j * g.W + col];
        double q = (kind == 0) ? tj - acc : fma((double)deg[j], tj, -acc);
        if (is_anchor[j]) q += xj;
        r = B[j * g.W + col] - q;
        rr = fma(r, r, rr);
        xx = fma(xj, xj, xx);
      }
      R[j * g.W + col] = r;
    }
  }
  cta_col_partial(rr, sh, partials, col, g.W, col < g.W);
  cta_col_partial(xx, sh, partials + (long long)g.row_blocks * g.W, col, g.W, col < g.W);
}

// (row block, column) partials of B.B
__global__ void __launch_bounds__(kCgThreads) k_col_dots(CgGeom g, const double* __restrict__ B,
                                                         double* __restrict__ partials) {
  __shared__ double sh[256];
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rl = threadIdx.x >> 5;
  const long long r0 = (long long)blockIdx.y * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  double s = 0.0;
  if (col < g.W)
    for (long long j = r0 + rl; j < r1; j += 8) {
      const double b = B[j * g.W + col];
      s = fma(b, b, s);
    }
  cta_col_partial(s, sh, partials, col, g.W, col < g.W);
}

// out[col] = sum of the partials.  With check (partials of ||R||^2, then of
// ||X||^2), a column is done when ||R||^2 <= rtol2 ||B||^2, or when an outer
// step reduced ||R|| by less than half (prev: the last step's ||R||^2) while
// ||R||^2 <= floor2 ||X||^2: the FP64 residual has reached what binary64 can
// resolve for that X (backward-error test of mixed-precision refinement);
// *active counts the columns still open
__global__ void k_refine_sum(CgGeom g, const double* __restrict__ partials, double* out,
                             int check, const double* __restrict__ bb, double rtol2,
                             double floor2, double* prev, int32_t* frozen, int32_t* active) {
  const int col = blockIdx.x;   // grid: one CTA per column
  const double s = col_sum(partials, g.row_blocks, g.W, col);
  double xx = 0.0;
  if (check) xx = col_sum(partials + (long long)g.row_blocks * g.W, g.row_blocks, g.W, col);
  if (threadIdx.x == 0) {
    if (check) {
      if (!frozen[col]) {
        out[col] = s;
        const bool stalled = s > 0.25 * prev[col] && s <= floor2 * xx;
        if (s <= rtol2 * bb[col] || stalled) frozen[col] = 1;
        prev[col] = s;
      }
      if (!frozen[col]) atomicAdd(active, 1);
    } else {
      out[col] = s;
    }
  }
}

__global__ void k_fill_d(double* p, int count, double v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_refine_add(const float* __restrict__ D, long long count, double* __restrict__ X) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    X[e] += (double)D[e];
}

__global__ void k_refine_iters(const int32_t* __restrict__ it, int W, int32_t* total) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < W; c += gridDim.x * blockDim.x)
    total[c] += it[c];
}

void refine_col_norms(const CgGeom& g, const double* B, double* partials, double* out,
                      cudaStream_t s, Launches& L) {
  dim3 grid((g.W + 31) / 32, g.row_blocks);
  k_col_dots<<<grid, kCgThreads, 0, s>>>(g, B, partials);
  k_refine_sum<<<g.W, 256, 0, s>>>(g, partials, out, 0, nullptr, 0.0, 0.0, nullptr,
                                             nullptr, nullptr);
  L.add(2);
}

void refine_reset(double* prev, int W, cudaStream_t s, Launches& L) {
  k_fill_d<<<(W + 255) / 256, 256, 0, s>>>(prev, W, 1e300);
  L.add(1);
}

void refine_residual(const CgGeom& g, const int32_t* row_ptr, const int32_t* col_idx,
                     const int32_t* deg, const double* inv_d, const uint8_t* is_anchor, int kind,
                     const double* X, const double* B, double* T, double* R, int32_t* frozen,
                     double* partials, const double* bb, double rtol, double floor, double* prev,
                     double* rr, int32_t* active, cudaStream_t s, Launches& L) {
  dim3 grid((g.W + 31) / 32, g.row_blocks);
  k_cg_L<double><<<grid, kCgThreads, 0, s>>>(g, row_ptr, col_idx, deg, inv_d, kind, X, T, frozen);
  k_refine_residual<<<grid, kCgThreads, 0, s>>>(g, row_ptr, col_idx, deg, inv_d, kind, is_anchor,
                                                T, X, B, R, frozen, partials);
  cudaMemsetAsync(active, 0, sizeof(int32_t), s);
  k_refine_sum<<<g.W, 256, 0, s>>>(g, partials, rr, 1, bb, rtol * rtol, floor * floor,
                                             prev, frozen, active);
  L.add(3);
}

__global__ void k_refine_targets(const double* __restrict__ rr, const double* __restrict__ bb,
                                 const int32_t* __restrict__ frozen, int W, double rtol,
                                 double inner, double* __restrict__ t2, double* cg_bb) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < W; c += gridDim.x * blockDim.x) {
    double t = 0.5;
    if (!frozen[c] && rr[c] > 0.0) t = fmin(0.5, fmax(inner, 0.8 * rtol * sqrt(bb[c] / rr[c])));
    const double q = frozen[c] ? 1.0 : (t / inner) * (t / inner);
    t2[c] = q;
    if (cg_bb) cg_bb[c] *= q;
  }
}

void refine_targets(const double* rr, const double* bb, const int32_t* frozen, int W, double rtol,
                    double inner_rtol, double* t2, double* cg_bb, cudaStream_t s, Launches& L) {
  k_refine_targets<<<(W + 255) / 256, 256, 0, s>>>(rr, bb, frozen, W, rtol, inner_rtol, t2, cg_bb);
  L.add(1);
}

void refine_update(const float* D, long long count, double* X, const int32_t* iters, int W,
                   int32_t* total, cudaStream_t s, Launches& L) {
  k_refine_add<<<(int)std::min<long long>((count + 255) / 256, 152 * 16), 256, 0, s>>>(D, count,
                                                                                      X);
  k_refine_iters<<<(W + 255) / 256, 256, 0, s>>>(iters, W, total);
  L.add(2);
}

// out[e] = (double) X[e]
__global__ void k_widen(const float* __restrict__ X, long long count, double* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (double)X[e];
}

// out[e] = (float) X[e]
__global__ void k_narrow(const double* __restrict__ X, long long count, float* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (float)X[e];
}

void narrow(const double* X, long long count, float* out, cudaStream_t s, Launches& L) {
  int grid = (int)std::min<long long>((count + 255) / 256, 152 * 32);
  k_narrow<<<std::max(grid, 1), 256, 0, s>>>(X, count, out);
  L.add(1);
}

void widen(const float* X, long long count, double* out, cudaStream_t s, Launches& L) {
  int grid = (int)std::min<long long>((count + 255) / 256, 152 * 32);
  k_widen<<<std::max(grid, 1), 256, 0, s>>>(X, count, out);
  L.add(1);
}

const char* const kCgKernelNames[kCgKernels] = {"k_cg_L", "k_cg_LT", "k_cg_alpha",
                                                "k_cg_update", "k_cg_beta", "k_cg_dir"};

// B[anchor a][coord_cols + f] += Ahat[a][f]   (P^T a^ for one coordinate block)
__global__ void k_scatter_anchor_rhs(double* B, const double* __restrict__ Ahat,
                                     const int32_t* __restrict__ anchors, int n_c, int F, int W,
                                     int coord_cols) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n_c * F;
       e += (long long)gridDim.x * blockDim.x) {
    long long a = e / F, f = e % F;
    B[(long long)anchors[a] * W + coord_cols + f] += Ahat[e];
  }
}

// E[i][c*k + r] = C'_c[r][i] for c < 3, r < k; E[i][3k + a] = 0   (E: [n][Wc])
__global__ void k_factored_rhs(const double* __restrict__ Cdeq, int k, int n, int Wc,
                               double* __restrict__ E) {
  const long long total = (long long)n * Wc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long i = e / Wc;
    int col = (int)(e % Wc);
    double v = 0.0;
    if (col < 3 * k) {
      int c = col / k, r = col % k;
      v = Cdeq[((long long)c * k + r) * n + i];
    }
    E[e] = v;
  }
}

void factored_rhs(const double* Cdeq, int k, int n, int Wc, double* E, cudaStream_t s,
                  Launches& L) {
  long long total = (long long)n * Wc;
  int grid = (int)std::min<long long>((total + 255) / 256, 152 * 32);
  k_factored_rhs<<<grid, 256, 0, s>>>(Cdeq, k, n, Wc, E);
  L.add(1);
}

// B[anchor a][col0 + a] += 1   (the columns of P^T)
__global__ void k_unit_anchor_columns(double* B, const int32_t* __restrict__ anchors, int n_c,
                                      int Wc, int col0) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n_c; a += gridDim.x * blockDim.x)
    B[(long long)anchors[a] * Wc + col0 + a] += 1.0;
}

void unit_anchor_columns(double* B, const int32_t* anchors, int n_c, int Wc, int col0,
                         cudaStream_t s, Launches& L) {
  if (n_c <= 0) return;
  k_unit_anchor_columns<<<(n_c + 255) / 256, 256, 0, s>>>(B, anchors, n_c, Wc, col0);
  L.add(1);
}

void scatter_anchor_rhs(double* B, const double* Ahat, const int32_t* anchors, int n_c, int F,
                        int W, int coord_cols, cudaStream_t s, Launches& L) {
  if (n_c <= 0) return;
  long long tot = (long long)n_c * F;
  int grid = (int)std::min<long long>((tot + 255) / 256, 1024);
  k_scatter_anchor_rhs<<<grid, 256, 0, s>>>(B, Ahat, anchors, n_c, F, W, coord_cols);
  L.add(1);
}

}  // namespace mc
