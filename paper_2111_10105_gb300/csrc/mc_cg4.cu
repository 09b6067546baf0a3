// FP32 decoder CG with four columns per thread (the mixed-precision modes).
//
// Same iteration, reduction order and results as the scalar FP32 kernels of
// mc_cg.cu, for column counts W divisible by 4: every load and store moves a
// float4 (512 bytes per warp per vertex row instead of 128), which keeps
// enough bytes in flight per SM for these HBM-bound sweeps.  A CTA covers
// LANES column lanes (4 * LANES columns) x 8 row lanes, LANES = 32, 16 or 8
// (256, 128 or 64 threads), chosen per column count to leave the fewest
// columns idle: each column keeps the same row lanes and the same fixed
// reduction order at every width, so the width does not change the results.
// A group of four columns is skipped only when all four have converged; a
// converged column inside an active group is recomputed harmlessly (its
// alpha and beta are 0, its dot products unused).
#include <algorithm>
#include <type_traits>

#include "mc_internal.cuh"

namespace mc {

namespace {

constexpr int kRowLanes = 8;

struct Dot2 {   // compensated FP32 dot product (TwoProduct + TwoSum)
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// the thread's column lane and row lane
template <int LANES>
__device__ __forceinline__ int col_lane() { return threadIdx.x % LANES; }
template <int LANES>
__device__ __forceinline__ int row_lane() { return threadIdx.x / LANES; }
template <int LANES>
__device__ __forceinline__ int first_col(int bx) {
  return bx * (4 * LANES) + col_lane<LANES>() * 4;
}

// combine the 8 row lanes' partial sums of this CTA's 4 * LANES columns, fixed order
template <int LANES>
__device__ __forceinline__ void cta_partials4(const double v[4], double (*sh)[4 * LANES + 1],
                                              double* out, int W, int col0, bool valid, int by) {
  const int lane = col_lane<LANES>(), rl = row_lane<LANES>();
#pragma unroll
  for (int c = 0; c < 4; ++c) sh[rl][lane * 4 + c] = v[c];
  __syncthreads();
  if (rl == 0 && valid) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double s = sh[0][lane * 4 + c];
#pragma unroll
      for (int r = 1; r < kRowLanes; ++r) s += sh[r][lane * 4 + c];
      out[(long long)by * W + col0 + c] = s;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ bool group_done(const int32_t* done, int col0) {
  return done[col0] && done[col0 + 1] && done[col0 + 2] && done[col0 + 3];
}

template <int LANES>
__global__ void __launch_bounds__(LANES * kRowLanes) k4_init(CgGeom g, const double* __restrict__ B,
                                                             float* __restrict__ X,
                                                             float* __restrict__ R,
                                                             float* __restrict__ P,
                                                             const float* __restrict__ inv_diag,
                                                             double* __restrict__ partials) {
  __shared__ double sh[kRowLanes][4 * LANES + 1];
  const int col0 = first_col<LANES>(blockIdx.x);
  const int rl = row_lane<LANES>();
  const bool valid = col0 < g.W;
  const long long r0 = (long long)blockIdx.y * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  Dot2 rz[4], bb[4];
  if (valid) {
    for (long long i = r0 + rl; i < r1; i += kRowLanes) {
      const long long e = i * g.W + col0;
      const float d = inv_diag[i];
      float b[4], z[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        b[c] = (float)B[e + c];
        z[c] = b[c] * d;
        rz[c].add(b[c], z[c]);
        bb[c].add(b[c], b[c]);
      }
      st4(X + e, make_float4(0.f, 0.f, 0.f, 0.f));
      st4(R + e, make_float4(b[0], b[1], b[2], b[3]));
      st4(P + e, make_float4(z[0], z[1], z[2], z[3]));
    }
  }
  const long long plane = (long long)g.row_blocks * g.W;
  double v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = rz[c].value();
  cta_partials4<LANES>(v, sh, partials, g.W, col0, valid, blockIdx.y);
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = bb[c].value();
  cta_partials4<LANES>(v, sh, partials + plane, g.W, col0, valid, blockIdx.y);
}

// sum of the neighbours' float4 rows, ascending, loaded four rows at a time
__device__ __forceinline__ float4 gather4(const float* __restrict__ V, const int32_t* __restrict__ ci,
                                          int b, int e, int W, int col0) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  int p = b;
  for (; p + 4 <= e; p += 4) {
    const float4 v0 = ld4(V + (long long)ci[p] * W + col0);
    const float4 v1 = ld4(V + (long long)ci[p + 1] * W + col0);
    const float4 v2 = ld4(V + (long long)ci[p + 2] * W + col0);
    const float4 v3 = ld4(V + (long long)ci[p + 3] * W + col0);
    acc.x += v0.x; acc.y += v0.y; acc.z += v0.z; acc.w += v0.w;
    acc.x += v1.x; acc.y += v1.y; acc.z += v1.z; acc.w += v1.w;
    acc.x += v2.x; acc.y += v2.y; acc.z += v2.z; acc.w += v2.w;
    acc.x += v3.x; acc.y += v3.y; acc.z += v3.z; acc.w += v3.w;
  }
  for (; p < e; ++p) {
    const float4 v = ld4(V + (long long)ci[p] * W + col0);
    acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
  }
  return acc;
}

// The CTA's slice of the adjacency, staged in shared memory when the tile
// geometry allows it (g.csr_cap > 0): row offsets relative to the block's
// first entry, then the column indices.  All threads of the CTA take part.
// Each gather then finds its neighbour indices in shared memory instead of
// behind two dependent global loads.  rp is indexed by row - r0.
struct CsrSlice {
  const int32_t* rp;
  const int32_t* ci;
};

__device__ __forceinline__ CsrSlice stage_csr(const CgGeom& g, const int32_t* __restrict__ row_ptr,
                                              const int32_t* __restrict__ col_idx, long long r0,
                                              long long r1, int32_t* smem) {
  if (g.csr_cap > 0) {
    const int base = row_ptr[r0];
    const int cnt = row_ptr[r1] - base;
    if (cnt <= g.csr_cap) {                 // the same for every thread of the CTA
      int32_t* s_rp = smem;
      int32_t* s_ci = smem + g.rows_per_block + 1;
      const int nr = (int)(r1 - r0);
      for (int t = threadIdx.x; t <= nr; t += blockDim.x) s_rp[t] = row_ptr[r0 + t] - base;
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) s_ci[t] = col_idx[base + t];
      __syncthreads();
      return CsrSlice{s_rp, s_ci};
    }
  }
  return CsrSlice{row_ptr + r0, col_idx};
}

// T = L P (Eq. 4) or T = D^-1 L P (Eq. 3) over one (column tile bx, row block by)
template <int LANES>
__device__ __forceinline__ void k4_L_body(const CgGeom& g, int bx, int by,
                                          const int32_t* __restrict__ row_ptr,
                                          const int32_t* __restrict__ col_idx,
                                          const int32_t* __restrict__ deg,
                                          const float* __restrict__ inv_d, int kind,
                                          const float* __restrict__ P, float* __restrict__ T,
                                          const int32_t* __restrict__ done, int32_t* smem) {
  const int col0 = first_col<LANES>(bx);
  const int rl = row_lane<LANES>();
  const long long r0 = (long long)by * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  const CsrSlice cs = stage_csr(g, row_ptr, col_idx, r0, r1, smem);
  if (col0 >= g.W || group_done(done, col0)) return;
  for (long long i = r0 + rl; i < r1; i += kRowLanes) {
    const float4 s = gather4(P, cs.ci, cs.rp[i - r0], cs.rp[i - r0 + 1], g.W, col0);
    const float4 p = ld4(P + i * g.W + col0);
    float4 t;
    if (kind == 0) {   // Y = D^-1 (L P): the second pass then needs no weights
      const float w = inv_d[i], a = -w;
      t = make_float4(w * fmaf(a, s.x, p.x), w * fmaf(a, s.y, p.y), w * fmaf(a, s.z, p.z),
                      w * fmaf(a, s.w, p.w));
    } else {
      const float d = (float)deg[i];
      t = make_float4(fmaf(d, p.x, -s.x), fmaf(d, p.y, -s.y), fmaf(d, p.z, -s.z),
                      fmaf(d, p.w, -s.w));
    }
    st4(T + i * g.W + col0, t);
  }
}

// (the gathers are latency-bound: launched for a full SM of 2,048 threads, at
// most 32 registers, a few spilled; measured 7% faster per iteration than
// their natural 34 / 44 registers)
template <int LANES>
__global__ void __launch_bounds__(LANES * kRowLanes, 2048 / (LANES * kRowLanes)) k4_L(CgGeom g,
                                                          const int32_t* __restrict__ row_ptr,
                                                          const int32_t* __restrict__ col_idx,
                                                          const int32_t* __restrict__ deg,
                                                          const float* __restrict__ inv_d,
                                                          int kind, const float* __restrict__ P,
                                                          float* __restrict__ T,
                                                          const int32_t* __restrict__ done) {
  extern __shared__ int32_t smem_csr[];
  k4_L_body<LANES>(g, blockIdx.x, blockIdx.y, row_ptr, col_idx, deg, inv_d, kind, P, T, done,
                   smem_csr);
}

// Q = L^T L P + [anchor] P = K T + [anchor] P and the pAp partials over one
// (column tile, row block), K = D - A
template <int LANES>
__device__ __forceinline__ void k4_LT_body(const CgGeom& g, int bx, int by,
                                           const int32_t* __restrict__ row_ptr,
                                           const int32_t* __restrict__ col_idx,
                                           const int32_t* __restrict__ deg,
                                           const float* __restrict__ inv_d, int kind,
                                           const uint8_t* __restrict__ is_anchor,
                                           const float* __restrict__ T,
                                           const float* __restrict__ P, float* __restrict__ Q,
                                           const int32_t* __restrict__ done,
                                           double* __restrict__ partials,
                                           double (*sh)[4 * LANES + 1]) {
  // (the CSR slice stays in global memory here: staging it costs this kernel
  // four registers and an occupancy step, more than the shorter load chain
  // saves; measured on the 99,856-vertex grid)
  const int col0 = first_col<LANES>(bx);
  const int rl = row_lane<LANES>();
  const bool valid = col0 < g.W && !group_done(done, col0);
  const long long r0 = (long long)by * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  Dot2 pap[4];
  if (valid) {
    for (long long j = r0 + rl; j < r1; j += kRowLanes) {
      // L^T T = K T (Eq. 4, K = D - A) or, with L = D^-1 K (Eq. 3) and T holding
      // Y = D^-1 L P, L^T L P = K Y: the same unweighted neighbour sum for both
      const int b = row_ptr[j], e = row_ptr[j + 1];
      const float4 a = gather4(T, col_idx, b, e, g.W, col0);
      const float4 t = ld4(T + j * g.W + col0);
      const float4 p = ld4(P + j * g.W + col0);
      const float d = (float)deg[j];
      float q[4] = {fmaf(d, t.x, -a.x), fmaf(d, t.y, -a.y), fmaf(d, t.z, -a.z),
                    fmaf(d, t.w, -a.w)};
      if (is_anchor[j]) {
        q[0] += p.x; q[1] += p.y; q[2] += p.z; q[3] += p.w;
      }
      st4(Q + j * g.W + col0, make_float4(q[0], q[1], q[2], q[3]));
      pap[0].add(p.x, q[0]);
      pap[1].add(p.y, q[1]);
      pap[2].add(p.z, q[2]);
      pap[3].add(p.w, q[3]);
    }
  }
  double v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = pap[c].value();
  cta_partials4<LANES>(v, sh, partials, g.W, col0, col0 < g.W, by);
}

template <int LANES>
__global__ void __launch_bounds__(LANES * kRowLanes, 2048 / (LANES * kRowLanes)) k4_LT(CgGeom g,
                                                           const int32_t* __restrict__ row_ptr,
                                                           const int32_t* __restrict__ col_idx,
                                                           const int32_t* __restrict__ deg,
                                                           const float* __restrict__ inv_d,
                                                           int kind,
                                                           const uint8_t* __restrict__ is_anchor,
                                                           const float* __restrict__ T,
                                                           const float* __restrict__ P,
                                                           float* __restrict__ Q,
                                                           const int32_t* __restrict__ done,
                                                           double* __restrict__ partials) {
  __shared__ double sh[kRowLanes][4 * LANES + 1];
  k4_LT_body<LANES>(g, blockIdx.x, blockIdx.y, row_ptr, col_idx, deg, inv_d, kind, is_anchor, T,
                    P, Q, done, partials, sh);
}

// X += alpha P, R -= alpha Q and the rz / rr partials over one (column tile, row block)
template <int LANES>
__device__ __forceinline__ void k4_update_body(const CgGeom& g, int bx, int by,
                                               float* __restrict__ X, float* __restrict__ R,
                                               const float* __restrict__ P,
                                               const float* __restrict__ Q,
                                               const float* __restrict__ inv_diag,
                                               const double* __restrict__ alpha,
                                               const int32_t* __restrict__ done,
                                               double* __restrict__ partials,
                                               double (*sh)[4 * LANES + 1]) {
  const int col0 = first_col<LANES>(bx);
  const int rl = row_lane<LANES>();
  const bool valid = col0 < g.W && !group_done(done, col0);
  const long long r0 = (long long)by * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  Dot2 rz[4], rr[4];
  if (valid) {
    const float a0 = (float)alpha[col0], a1 = (float)alpha[col0 + 1];
    const float a2 = (float)alpha[col0 + 2], a3 = (float)alpha[col0 + 3];
    auto step = [&](long long e, float4 x, float4 r, float4 p, float4 q, float d) {
      st4(X + e, make_float4(fmaf(a0, p.x, x.x), fmaf(a1, p.y, x.y), fmaf(a2, p.z, x.z),
                             fmaf(a3, p.w, x.w)));
      const float4 rn = make_float4(fmaf(-a0, q.x, r.x), fmaf(-a1, q.y, r.y), fmaf(-a2, q.z, r.z),
                                    fmaf(-a3, q.w, r.w));
      st4(R + e, rn);
      rz[0].add(rn.x, rn.x * d); rr[0].add(rn.x, rn.x);
      rz[1].add(rn.y, rn.y * d); rr[1].add(rn.y, rn.y);
      rz[2].add(rn.z, rn.z * d); rr[2].add(rn.z, rn.z);
      rz[3].add(rn.w, rn.w * d); rr[3].add(rn.w, rn.w);
    };
    // two rows' loads in flight before either row's stores (rows in ascending order)
    const long long stride = (long long)kRowLanes * g.W;
    long long i = r0 + rl;
    for (; i + kRowLanes < r1; i += 2 * kRowLanes) {
      const long long e = i * g.W + col0;
      const float4 x0 = ld4(X + e), rv0 = ld4(R + e), p0 = ld4(P + e), q0 = ld4(Q + e);
      const float4 x1 = ld4(X + e + stride), rv1 = ld4(R + e + stride);
      const float4 p1 = ld4(P + e + stride), q1 = ld4(Q + e + stride);
      const float d0 = inv_diag[i], d1 = inv_diag[i + kRowLanes];
      step(e, x0, rv0, p0, q0, d0);
      step(e + stride, x1, rv1, p1, q1, d1);
    }
    if (i < r1) {
      const long long e = i * g.W + col0;
      step(e, ld4(X + e), ld4(R + e), ld4(P + e), ld4(Q + e), inv_diag[i]);
    }
  }
  const long long plane = (long long)g.row_blocks * g.W;
  double v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = rz[c].value();
  cta_partials4<LANES>(v, sh, partials, g.W, col0, col0 < g.W, by);
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = rr[c].value();
  cta_partials4<LANES>(v, sh, partials + plane, g.W, col0, col0 < g.W, by);
}

// (at most 64 registers: 1,024 resident threads per SM, each with two rows of
// loads in flight)
template <int LANES>
__global__ void __launch_bounds__(LANES * kRowLanes, 1024 / (LANES * kRowLanes))
    k4_update(CgGeom g, float* __restrict__ X, float* __restrict__ R,
              const float* __restrict__ P, const float* __restrict__ Q,
              const float* __restrict__ inv_diag, const double* __restrict__ alpha,
              const int32_t* __restrict__ done, double* __restrict__ partials) {
  __shared__ double sh[kRowLanes][4 * LANES + 1];
  k4_update_body<LANES>(g, blockIdx.x, blockIdx.y, X, R, P, Q, inv_diag, alpha, done, partials,
                        sh);
}

// P = D^-1 R + beta P over one (column tile, row block)
template <int LANES>
__device__ __forceinline__ void k4_dir_body(const CgGeom& g, int bx, int by,
                                            const float* __restrict__ R, float* __restrict__ P,
                                            const float* __restrict__ inv_diag,
                                            const double* __restrict__ beta,
                                            const int32_t* __restrict__ done) {
  const int col0 = first_col<LANES>(bx);
  const int rl = row_lane<LANES>();
  if (col0 >= g.W || group_done(done, col0)) return;
  const float b0 = (float)beta[col0], b1 = (float)beta[col0 + 1];
  const float b2 = (float)beta[col0 + 2], b3 = (float)beta[col0 + 3];
  const long long r0 = (long long)by * g.rows_per_block;
  const long long r1 = std::min<long long>(g.n, r0 + g.rows_per_block);
  for (long long i = r0 + rl; i < r1; i += kRowLanes) {
    const long long e = i * g.W + col0;
    const float4 r = ld4(R + e), p = ld4(P + e);
    const float d = inv_diag[i];
    st4(P + e, make_float4(fmaf(b0, p.x, r.x * d), fmaf(b1, p.y, r.y * d), fmaf(b2, p.z, r.z * d),
                           fmaf(b3, p.w, r.w * d)));
  }
}

template <int LANES>
__global__ void __launch_bounds__(LANES * kRowLanes) k4_dir(CgGeom g, const float* __restrict__ R,
                                                            float* __restrict__ P,
                                                            const float* __restrict__ inv_diag,
                                                            const double* __restrict__ beta,
                                                            const int32_t* __restrict__ done) {
  k4_dir_body<LANES>(g, blockIdx.x, blockIdx.y, R, P, inv_diag, beta, done);
}

// ------------------------------------------------ grouped (work-table) kernels
// One CTA per item of a table: CTA i runs item i (CTAs past the table's
// current length return at once; the table only shrinks) with the same item
// body as the per-solve kernels and that solve's geometry and vectors, so
// every solve of the batch gets the results it gets alone (same row lanes,
// partials and reduction order).
constexpr int kGroupLanes = kGroupCols / 4;

__global__ void __launch_bounds__(kGroupLanes * kRowLanes) k4g_L(const CgSeq* __restrict__ seqs,
                                                                  const int4* __restrict__ items,
                                                                  const int* __restrict__ n_items) {
  extern __shared__ int32_t smem_csr[];
  if ((int)blockIdx.x >= *n_items) return;
  const int4 w = items[blockIdx.x];
  const CgSeq& q = seqs[w.x];
  k4_L_body<kGroupLanes>(q.g, w.z, w.y, q.row_ptr, q.col_idx, q.deg, q.inv_d, q.kind, q.P, q.T,
                         q.done, smem_csr);
}

__global__ void __launch_bounds__(kGroupLanes * kRowLanes) k4g_LT(const CgSeq* __restrict__ seqs,
                                                                   const int4* __restrict__ items,
                                                                   const int* __restrict__ n_items) {
  __shared__ double sh[kRowLanes][4 * kGroupLanes + 1];
  if ((int)blockIdx.x >= *n_items) return;
  const int4 w = items[blockIdx.x];
  const CgSeq& q = seqs[w.x];
  k4_LT_body<kGroupLanes>(q.g, w.z, w.y, q.row_ptr, q.col_idx, q.deg, q.inv_d, q.kind,
                          q.is_anchor, q.T, q.P, q.Q, q.done, q.partials, sh);
}

__global__ void __launch_bounds__(kGroupLanes * kRowLanes, 1024 / (kGroupLanes * kRowLanes))
    k4g_update(const CgSeq* __restrict__ seqs, const int4* __restrict__ items,
               const int* __restrict__ n_items) {
  __shared__ double sh[kRowLanes][4 * kGroupLanes + 1];
  if ((int)blockIdx.x >= *n_items) return;
  const int4 w = items[blockIdx.x];
  const CgSeq& q = seqs[w.x];
  k4_update_body<kGroupLanes>(q.g, w.z, w.y, q.X, q.R, q.P, q.Q, q.inv_diag, q.alpha, q.done,
                              q.partials, sh);
}

__global__ void __launch_bounds__(kGroupLanes * kRowLanes) k4g_dir(const CgSeq* __restrict__ seqs,
                                                                    const int4* __restrict__ items,
                                                                    const int* __restrict__ n_items) {
  if ((int)blockIdx.x >= *n_items) return;
  const int4 w = items[blockIdx.x];
  const CgSeq& q = seqs[w.x];
  k4_dir_body<kGroupLanes>(q.g, w.z, w.y, q.R, q.P, q.inv_diag, q.beta, q.done);
}

}  // namespace

size_t cg4_grouped_smem(const CgGeom& g) {
  return g.csr_cap > 0 ? sizeof(int32_t) * (g.rows_per_block + 1 + g.csr_cap) : 0;
}

void cg4_grouped_iteration(const CgSeq* seqs, const int4* items, const int* n_items,
                           const int2* cols, const int* n_cols, int grid_rows, int grid_cols,
                           size_t smem, cudaStream_t s, Launches& L) {
  constexpr int T = kGroupLanes * kRowLanes;
  k4g_L<<<grid_rows, T, smem, s>>>(seqs, items, n_items);
  k4g_LT<<<grid_rows, T, 0, s>>>(seqs, items, n_items);
  cgg_alpha(seqs, cols, n_cols, grid_cols, s);
  k4g_update<<<grid_rows, T, 0, s>>>(seqs, items, n_items);
  cgg_beta(seqs, cols, n_cols, grid_cols, s);
  k4g_dir<<<grid_rows, T, 0, s>>>(seqs, items, n_items);
  L.add(6);
}

// column lanes per CTA for W columns: the fewest idle columns, the widest tile on ties
static int cg4_lanes(int W) {
  int best = 32;
  long long best_idle = -1;
  for (int lanes : {32, 16, 8}) {
    const long long cols = 4LL * lanes;
    const long long idle = (W + cols - 1) / cols * cols - W;
    if (best_idle < 0 || idle < best_idle) {
      best = lanes;
      best_idle = idle;
    }
  }
  return best;
}

template <typename Fn>
static void with_lanes(int W, Fn&& fn) {
  switch (cg4_lanes(W)) {
    case 32: fn(std::integral_constant<int, 32>()); break;
    case 16: fn(std::integral_constant<int, 16>()); break;
    default: fn(std::integral_constant<int, 8>()); break;
  }
}

template <int LANES>
static dim3 grid4(const CgGeom& g) {
  return dim3((g.W + 4 * LANES - 1) / (4 * LANES), g.row_blocks);
}

bool cg4_applies(int W, int single) { return single && (W % 4) == 0; }

void cg4_init(const CgGeom& g, const double* B, float* X, float* R, float* P,
              const float* inv_diag, double* partials, cudaStream_t s) {
  with_lanes(g.W, [&](auto lanes) {
    constexpr int LN = decltype(lanes)::value;
    k4_init<LN><<<grid4<LN>(g), LN * kRowLanes, 0, s>>>(g, B, X, R, P, inv_diag, partials);
  });
}

void cg4_op(const CgGeom& g, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* deg,
            const float* inv_d, int kind, const uint8_t* is_anchor, const float* P, float* T,
            float* Q, const int32_t* done, double* partials, cudaStream_t s, cudaEvent_t* ev) {
  const size_t smem = g.csr_cap > 0 ? sizeof(int32_t) * (g.rows_per_block + 1 + g.csr_cap) : 0;
  with_lanes(g.W, [&](auto lanes) {
    constexpr int LN = decltype(lanes)::value;
    k4_L<LN><<<grid4<LN>(g), LN * kRowLanes, smem, s>>>(g, row_ptr, col_idx, deg, inv_d, kind,
                                                        P, T, done);
    if (ev) cudaEventRecord(ev[1], s);
    k4_LT<LN><<<grid4<LN>(g), LN * kRowLanes, 0, s>>>(g, row_ptr, col_idx, deg, inv_d, kind,
                                                      is_anchor, T, P, Q, done, partials);
  });
}

void cg4_update(const CgGeom& g, float* X, float* R, const float* P, const float* Q,
                const float* inv_diag, const double* alpha, const int32_t* done,
                double* partials, cudaStream_t s) {
  with_lanes(g.W, [&](auto lanes) {
    constexpr int LN = decltype(lanes)::value;
    k4_update<LN><<<grid4<LN>(g), LN * kRowLanes, 0, s>>>(g, X, R, P, Q, inv_diag, alpha, done,
                                                          partials);
  });
}

void cg4_dir(const CgGeom& g, const float* R, float* P, const float* inv_diag, const double* beta,
             const int32_t* done, cudaStream_t s) {
  with_lanes(g.W, [&](auto lanes) {
    constexpr int LN = decltype(lanes)::value;
    k4_dir<LN><<<grid4<LN>(g), LN * kRowLanes, 0, s>>>(g, R, P, inv_diag, beta, done);
  });
}

}  // namespace mc
