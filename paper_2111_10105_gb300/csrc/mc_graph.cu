// Mesh graph kernels: CSR adjacency from triangles (Section II, Eq. 2), the
// anchor set (Section III, before Eq. 12), and the Laplacian products of
// Eq. 3/4 (delta coordinates) and of the decoder's normal equations.
#include <algorithm>

#include "mc_internal.cuh"

namespace mc {

// ------------------------------------------------------------ exclusive scan
// Three passes: per-block scan of 2048 items with block totals, a
// single-block scan of the totals (looping with a carry), and the add-back.
static constexpr int kScanBlock = 1024;
static constexpr int kScanItems = 2 * kScanBlock;

size_t scan_tmp_elems(int n) { return (size_t)(n / kScanItems + 2); }

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t* sh, int32_t* total) {
  // Hillis-Steele on warp sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  int32_t incl = x + (warp > 0 ? sh[warp - 1] : 0);
  if (total) *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return incl - v;
}

__global__ void k_scan_blocks(const int32_t* in, int32_t* out, int n, int32_t* block_sums) {
  __shared__ int32_t sh[32];
  long long base = (long long)blockIdx.x * kScanItems;
  long long i0 = base + 2 * threadIdx.x;
  int32_t a = (i0 < n) ? in[i0] : 0;
  int32_t b = (i0 + 1 < n) ? in[i0 + 1] : 0;
  int32_t tot;
  int32_t ex = block_excl_scan(a + b, sh, &tot);
  if (i0 < n) out[i0] = ex;
  if (i0 + 1 < n) out[i0 + 1] = ex + a;
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int32_t* sums, int nb, int32_t* grand_total_out) {
  __shared__ int32_t sh[32];
  int32_t carry = 0;
  for (int base = 0; base < nb; base += kScanBlock) {
    int i = base + threadIdx.x;
    int32_t v = (i < nb) ? sums[i] : 0;
    int32_t tot;
    int32_t ex = block_excl_scan(v, sh, &tot);
    if (i < nb) sums[i] = ex + carry;
    carry += tot;
  }
  if (threadIdx.x == 0) *grand_total_out = carry;
}

__global__ void k_scan_add(int32_t* out, int n, const int32_t* sums) {
  long long i = (long long)blockIdx.x * kScanItems + threadIdx.x;
  int32_t add = sums[blockIdx.x];
  if (i < n) out[i] += add;
  if (i + kScanBlock < n) out[i + kScanBlock] += add;
}

void exclusive_scan_i32(const int32_t* in, int32_t* out, int n, int32_t* tmp, cudaStream_t s,
                        Launches& L) {
  int nb = (n + kScanItems - 1) / kScanItems;
  if (nb < 1) nb = 1;
  k_scan_blocks<<<nb, kScanBlock, 0, s>>>(in, out, n, tmp);
  k_scan_sums<<<1, kScanBlock, 0, s>>>(tmp, nb, out + n);
  k_scan_add<<<nb, kScanBlock, 0, s>>>(out, n, tmp);
  L.add(3);
}

// ------------------------------------------------------------ CSR build
__device__ __forceinline__ bool tri_ok(int a, int b, int c, int n, uint32_t* status) {
  if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n) {
    atomicOr(status, ST_BAD_INDEX);
    return false;
  }
  if (a == b || b == c || a == c) {
    atomicOr(status, ST_DEGENERATE);
    return false;
  }
  return true;
}

__global__ void k_csr_count(const int32_t* tris, int T, int n, int32_t* raw_deg,
                            uint32_t* status) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T;
       t += (long long)gridDim.x * blockDim.x) {
    int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
    if (!tri_ok(a, b, c, n, status)) continue;
    atomicAdd(&raw_deg[a], 2);
    atomicAdd(&raw_deg[b], 2);
    atomicAdd(&raw_deg[c], 2);
  }
}

__global__ void k_csr_fill(const int32_t* tris, int T, int n, const int32_t* raw_off,
                           int32_t* cursor, int32_t* raw_col) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T;
       t += (long long)gridDim.x * blockDim.x) {
    int v[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
    if (v[0] < 0 || v[1] < 0 || v[2] < 0 || v[0] >= n || v[1] >= n || v[2] >= n) continue;
    if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) continue;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      int me = v[e];
      int p = raw_off[me] + atomicAdd(&cursor[me], 2);
      raw_col[p] = v[(e + 1) % 3];
      raw_col[p + 1] = v[(e + 2) % 3];
    }
  }
}

// One thread per row: insertion sort of the row's raw neighbour list in
// place, duplicates removed; the unique, ascending list is left at the front
// of the row's raw segment and its length is d_i.
__global__ void k_csr_sort_unique(const int32_t* raw_off, int32_t* raw_col, int n,
                                  int32_t* deg, uint32_t* status) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int b = raw_off[i], e = raw_off[i + 1];
    for (int p = b + 1; p < e; ++p) {
      int v = raw_col[p];
      int q = p - 1;
      while (q >= b && raw_col[q] > v) {
        raw_col[q + 1] = raw_col[q];
        --q;
      }
      raw_col[q + 1] = v;
    }
    int u = 0;
    for (int p = b; p < e; ++p) {
      if (u == 0 || raw_col[b + u - 1] != raw_col[p]) raw_col[b + u++] = raw_col[p];
    }
    deg[i] = u;
    if (u == 0) atomicOr(status, ST_ISOLATED);
  }
}

__global__ void k_csr_compact(const int32_t* raw_off, const int32_t* raw_col,
                              const int32_t* row_ptr, int32_t* col_idx, int n) {
  // one warp per row
  long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = w; i < n; i += nw) {
    int b = raw_off[i], o = row_ptr[i], d = row_ptr[i + 1] - o;
    for (int j = lane; j < d; j += 32) col_idx[o + j] = raw_col[b + j];
  }
}

static int grid_for(long long work, int block, int max_blocks = 152 * 16) {
  long long g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

void build_csr(const int32_t* tris, int T, int n, CsrBuildTmp& t, int32_t* row_ptr,
               int32_t* /*unused*/, int32_t* deg, uint32_t* status, cudaStream_t s,
               Launches& L) {
  cudaMemsetAsync(t.raw_deg, 0, sizeof(int32_t) * n, s);
  cudaMemsetAsync(t.cursor, 0, sizeof(int32_t) * n, s);
  k_csr_count<<<grid_for(T, 256), 256, 0, s>>>(tris, T, n, t.raw_deg, status);
  exclusive_scan_i32(t.raw_deg, t.raw_off, n, t.scan_tmp, s, L);
  k_csr_fill<<<grid_for(T, 256), 256, 0, s>>>(tris, T, n, t.raw_off, t.cursor, t.raw_col);
  k_csr_sort_unique<<<grid_for(n, 128), 128, 0, s>>>(t.raw_off, t.raw_col, n, deg, status);
  exclusive_scan_i32(deg, row_ptr, n, t.scan_tmp, s, L);
  L.add(3);
}

void compact_csr(const CsrBuildTmp& t, const int32_t* row_ptr, int32_t* col_idx, int n,
                 cudaStream_t s, Launches& L) {
  k_csr_compact<<<grid_for((long long)n * 32, 256), 256, 0, s>>>(t.raw_off, t.raw_col, row_ptr,
                                                                 col_idx, n);
  L.add(1);
}

// ------------------------------------------------------------ anchors
// The n_c vertices with the smallest (key_i, i), key_i = splitmix64 output i
// of seed ^ kAnchorSalt, returned in ascending index order.  One CTA:
// a 64-step binary search for the n_c-th smallest key K (smallest K with
// #{key <= K} >= n_c), then an ordered compaction of {key < K} plus the
// lowest-index vertices with key == K.
__device__ __forceinline__ long long block_sum_ll(long long v, long long* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  long long t = 0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    sh[32] = t;
  }
  __syncthreads();
  t = sh[32];
  __syncthreads();
  return t;
}

__global__ void k_select_anchors(int n, int n_c, uint64_t seed, int32_t* anchors) {
  __shared__ long long shl[33];
  __shared__ int32_t shi[32];
  const uint64_t s = seed ^ kAnchorSalt;
  uint64_t lo = 0, hi = ~0ull;  // answer in [lo, hi]
  while (lo < hi) {
    uint64_t mid = lo + ((hi - lo) >> 1);
    long long c = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) c += (splitmix64_at(s, (uint64_t)i) <= mid);
    c = block_sum_ll(c, shl);
    if (c >= n_c) hi = mid; else lo = mid + 1;
  }
  const uint64_t K = lo;
  long long below = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) below += (splitmix64_at(s, (uint64_t)i) < K);
  below = block_sum_ll(below, shl);
  int32_t need_eq = (int32_t)(n_c - below);
  int32_t written = 0, eq_taken = 0;
  for (int base = 0; base < n; base += blockDim.x) {
    int i = base + threadIdx.x;
    uint64_t key = (i < n) ? splitmix64_at(s, (uint64_t)i) : ~0ull;
    int is_lt = (i < n) && key < K;
    int is_eq = (i < n) && key == K;
    int32_t tot_eq;
    int32_t ex_eq = block_excl_scan(is_eq, shi, &tot_eq);
    int take = is_lt || (is_eq && (eq_taken + ex_eq) < need_eq);
    int32_t tot_take;
    int32_t pos = block_excl_scan(take, shi, &tot_take);
    if (take) anchors[written + pos] = i;
    written += tot_take;
    eq_taken += tot_eq;
  }
}

void select_anchors(int n, int n_c, uint64_t seed, int32_t* anchors, cudaStream_t s,
                    Launches& L) {
  if (n_c <= 0) return;
  k_select_anchors<<<1, 1024, 0, s>>>(n, n_c, seed, anchors);
  L.add(1);
}

__global__ void k_check_anchors(const int32_t* a, int n_c, int n, uint32_t* status) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_c;
       i += (long long)gridDim.x * blockDim.x) {
    int v = a[i];
    bool bad = v < 0 || v >= n || (i > 0 && a[i - 1] >= v);
    if (bad) atomicOr(status, ST_BAD_ANCHORS);
  }
}

void check_anchors(const int32_t* anchors, int n_c, int n, uint32_t* status, cudaStream_t s,
                   Launches& L) {
  if (n_c <= 0) return;
  k_check_anchors<<<grid_for(n_c, 256), 256, 0, s>>>(anchors, n_c, n, status);
  L.add(1);
}

__global__ void k_mark_anchors(const int32_t* a, int n_c, uint8_t* is_anchor) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_c;
       i += (long long)gridDim.x * blockDim.x)
    is_anchor[a[i]] = 1;
}

void mark_anchors(const int32_t* anchors, int n_c, uint8_t* is_anchor, cudaStream_t s,
                  Launches& L) {
  if (n_c <= 0) return;
  k_mark_anchors<<<grid_for(n_c, 256), 256, 0, s>>>(anchors, n_c, is_anchor);
  L.add(1);
}

// inv_d_i = 1/d_i (kind 0) or 1 (kind 1, the weights of D - C's off-diagonal);
// inv_diag_m = 1 / diag(L^T L + P^T P):
//   kind 0: 1 + sum_{i in Psi_j} 1/d_i^2 + [j in N]
//   kind 1: d_j^2 + d_j + [j in N]
__global__ void k_vertex_scalars(const int32_t* row_ptr, const int32_t* col_idx,
                                 const int32_t* deg, const uint8_t* is_anchor, int n, int kind,
                                 double* inv_d, double* inv_diag_m) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    double dj = (double)deg[j];
    double m;
    if (kind == 0) {
      m = 1.0;
      for (int p = row_ptr[j]; p < row_ptr[j + 1]; ++p) {
        double di = (double)deg[col_idx[p]];
        m += 1.0 / (di * di);
      }
      inv_d[j] = 1.0 / dj;
    } else {
      m = dj * dj + dj;
      inv_d[j] = 1.0;
    }
    if (is_anchor[j]) m += 1.0;
    inv_diag_m[j] = 1.0 / m;
  }
}

void vertex_scalars_marked(const int32_t* row_ptr, const int32_t* col_idx, const int32_t* deg,
                           const uint8_t* is_anchor, int n, int kind, double* inv_d,
                           double* inv_diag_m, cudaStream_t s, Launches& L) {
  k_vertex_scalars<<<grid_for(n, 256), 256, 0, s>>>(row_ptr, col_idx, deg, is_anchor, n, kind,
                                                    inv_d, inv_diag_m);
  L.add(1);
}

// ------------------------------------------------------------ Laplacian rows
// Y = L X, X and Y [n][W].  Thread (row block, column): a CTA covers 32
// consecutive columns x RB rows; the neighbour sum runs in ascending column
// index order, then (kind 0) one correctly rounded division by d_i and one
// subtraction: the exact operation order the paper's Eq. 3 is evaluated in.
static constexpr int kLapRows = 8;

__global__ void __launch_bounds__(256) k_laplacian(const int32_t* __restrict__ row_ptr,
                                                   const int32_t* __restrict__ col_idx,
                                                   const int32_t* __restrict__ deg,
                                                   const double* __restrict__ X,
                                                   double* __restrict__ Y, int n, int W,
                                                   int kind) {
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rsub = threadIdx.x >> 5;  // 0..7
  if (col >= W) return;
  for (long long row0 = (long long)blockIdx.y * kLapRows * 8; row0 < n;
       row0 += (long long)gridDim.y * kLapRows * 8)
  for (int rr = 0; rr < kLapRows; ++rr) {
    long long i = row0 + rr * 8 + rsub;
    if (i >= n) break;
    int b = row_ptr[i], e = row_ptr[i + 1];
    double acc = 0.0;
    for (int p = b; p < e; ++p) acc = __dadd_rn(acc, X[(long long)col_idx[p] * W + col]);
    double xi = X[i * W + col];
    double out;
    if (kind == 0) {
      out = __dsub_rn(xi, __ddiv_rn(acc, (double)deg[i]));
    } else {
      out = __dsub_rn(__dmul_rn((double)deg[i], xi), acc);
    }
    Y[i * W + col] = out;
  }
}

void laplacian_rows(const int32_t* row_ptr, const int32_t* col_idx, const int32_t* deg,
                    const double* X, double* Y, int n, int W, int kind, cudaStream_t s,
                    Launches& L) {
  dim3 grid((W + 31) / 32, (unsigned)std::min<long long>((n + kLapRows * 8 - 1) / (kLapRows * 8), 65535));
  k_laplacian<<<grid, 256, 0, s>>>(row_ptr, col_idx, deg, X, Y, n, W, kind);
  L.add(1);
}

// B = L^T Y.  kind 0: (L^T y)_j = y_j - sum_{i in Psi_j} y_i / d_i (as an
// FMA chain with the precomputed 1/d_i); kind 1: L^T = L = D - C.
__global__ void __launch_bounds__(256) k_laplacian_t(const int32_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ col_idx,
                                                     const int32_t* __restrict__ deg,
                                                     const double* __restrict__ inv_d,
                                                     const double* __restrict__ Y,
                                                     double* __restrict__ B, int n, int W,
                                                     int kind) {
  const int col = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rsub = threadIdx.x >> 5;
  if (col >= W) return;
  for (long long row0 = (long long)blockIdx.y * kLapRows * 8; row0 < n;
       row0 += (long long)gridDim.y * kLapRows * 8)
  for (int rr = 0; rr < kLapRows; ++rr) {
    long long j = row0 + rr * 8 + rsub;
    if (j >= n) break;
    int b = row_ptr[j], e = row_ptr[j + 1];
    double acc = 0.0;
    if (kind == 0) {
      for (int p = b; p < e; ++p) {
        int i = col_idx[p];
        acc = fma(inv_d[i], Y[(long long)i * W + col], acc);
      }
      B[j * W + col] = Y[j * W + col] - acc;
    } else {
      for (int p = b; p < e; ++p) acc += Y[(long long)col_idx[p] * W + col];
      B[j * W + col] = (double)deg[j] * Y[j * W + col] - acc;
    }
  }
}

void laplacian_t_rows(const int32_t* row_ptr, const int32_t* col_idx, const int32_t* deg,
                      const double* inv_d, const double* Y, double* B, int n, int W, int kind,
                      cudaStream_t s, Launches& L) {
  dim3 grid((W + 31) / 32, (unsigned)std::min<long long>((n + kLapRows * 8 - 1) / (kLapRows * 8), 65535));
  k_laplacian_t<<<grid, 256, 0, s>>>(row_ptr, col_idx, deg, inv_d, Y, B, n, W, kind);
  L.add(1);
}

}  // namespace mc
