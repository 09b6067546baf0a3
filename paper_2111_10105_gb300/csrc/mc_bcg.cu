// Block conjugate gradients (O'Leary 1980) for the FP32 corrections of the
// refined decoder solve: M D = R with M = L^T L + P_a^T P_a the normal matrix
// of Eq. 12 and R the FP64 residual of the outer step.
//
// The right-hand sides are split into groups of up to 64 columns; a group
// shares one Krylov space.  Its search directions form an n x 64 block P,
// kept orthonormal, and every iteration takes the step that is optimal over
// the whole block:
//   Q = M P                               (the CG operator kernels)
//   G = P^T Q,  H = P^T R,  alpha = G^-1 H
//   X += P alpha,  R -= Q alpha
//   K = (D^-1 Q)^T R,  beta = -G^-1 K      (D = diag M, the Jacobi preconditioner)
//   P = orth(D^-1 R + P beta)              (CholeskyQR, twice)
// A group stops when each of its columns has ||r|| <= tol ||r_0|| (scaled per
// column by the refined solve's inner target).
//
// Precision.  The vectors are FP32.  The Gram matrices take FP32 products
// summed in FP32 over the rows one thread visits in a chunk of kChunkRows
// rows, and the chunks' partials are summed in FP64 in a fixed order
// (deterministic); the 64 x 64 factorisations and solves are FP64.  The
// block of new directions becomes nearly rank deficient as the columns
// converge and much of its information sits in directions of small Cholesky
// pivot, so the orthonormalisation needs Gram matrices accurate well beyond
// one FP32 rounding of a long sum.  Factorisations work on the unit-scaled
// matrix (D_s S D_s, D_s = diag(S)^-1/2), so a column of small norm is not
// mistaken for a dependent one; directions whose scaled pivot falls below
// kDropRel are dropped (their column of P is zero and the 64 x 64 solves
// leave them out).
#include <algorithm>
#include <cmath>

#include "mc_handle.cuh"

namespace mc {
namespace {

constexpr int kS = 64;            // columns per group
constexpr int kGramRows = 32;     // rows staged per step of the Gram kernel
constexpr int kChunkRows = 512;   // rows per Gram partial (128 FP32 products a thread)
constexpr int kMulRows = 128;     // rows per CTA of the block product
constexpr int kApplyCols = 4;     // right-hand sides per CTA of the 64 x 64 solves
constexpr int kCheck = 8;         // iterations between host convergence checks
constexpr double kDropRel = 1e-10;

// ---------------------------------------------------------------- Gram matrices
struct GramPair {
  const float* A;
  const float* B;
  float* part;   // [chunk][group][64][64]
};
struct GramArgs {
  GramPair pair[2];
  int npairs;
  const float* scale_a;   // rows of A multiplied by it (D^-1), or null
  float* sq_part;         // [chunk][W] column sums of squares of pair 0's B, or null
  int n, W, ngroups, rows_per_chunk;
  const int32_t* gdone;
};

// part[chunk][g][a][b] = sum over the chunk's rows r of A'[r][64g + a] B[r][64g + b].
// CTA (g * npairs + pair, chunk), 256 threads: four row slices of 64 threads,
// each thread an 8 x 8 tile of the 64 x 64 result over every fourth staged row.
__global__ void __launch_bounds__(256, 2) k_bgram(const GramArgs a) {
  __shared__ __align__(16) float buf[2 * kS * kS];   // staging, then the slices' sums
  __shared__ float sq_red[4][kS];
  float* sA = buf;
  float* sB = buf + kGramRows * kS;
  const int g = blockIdx.x / a.npairs, pi = blockIdx.x % a.npairs;
  if (a.gdone[g]) return;
  const GramPair pr = pi == 0 ? a.pair[0] : a.pair[1];
  const int chunk = blockIdx.y;
  const int c0 = g * kS, sg = min(kS, a.W - c0);
  const int t = threadIdx.x, slice = t >> 6, u = t & 63, ti = u >> 3, tj = u & 7;
  const long long r0 = (long long)chunk * a.rows_per_chunk;
  const long long r1 = min((long long)a.n, r0 + a.rows_per_chunk);
  const bool sq = a.sq_part != nullptr && pi == 0;
  float4 ra[2], rb[2];
  auto fetch = [&](long long base) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = t + q * 256, rr = e >> 4, c4 = (e & 15) * 4;
      const long long r = base + rr;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
      if (r < r1 && c4 < sg) {
        const long long o = r * a.W + c0 + c4;
        x = __ldg(reinterpret_cast<const float4*>(pr.A + o));
        y = __ldg(reinterpret_cast<const float4*>(pr.B + o));
        if (a.scale_a) {
          const float d = __ldg(a.scale_a + r);
          x.x *= d; x.y *= d; x.z *= d; x.w *= d;
        }
      }
      ra[q] = x;
      rb[q] = y;
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float sqacc = 0.f;
  fetch(r0);
  for (long long base = r0; base < r1; base += kGramRows) {
    __syncthreads();   // the previous tile is consumed
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = t + q * 256, rr = e >> 4, c4 = (e & 15) * 4;
      *reinterpret_cast<float4*>(sA + rr * kS + c4) = ra[q];
      *reinterpret_cast<float4*>(sB + rr * kS + c4) = rb[q];
    }
    __syncthreads();
    if (base + kGramRows < r1) fetch(base + kGramRows);   // in flight during the products
#pragma unroll 2
    for (int r = slice; r < kGramRows; r += 4) {
      const float4 a0 = *reinterpret_cast<const float4*>(sA + r * kS + 8 * ti);
      const float4 a1 = *reinterpret_cast<const float4*>(sA + r * kS + 8 * ti + 4);
      const float4 b0 = *reinterpret_cast<const float4*>(sB + r * kS + 8 * tj);
      const float4 b1 = *reinterpret_cast<const float4*>(sB + r * kS + 8 * tj + 4);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (sq)
      for (int r = slice; r < kGramRows; r += 4) {
        const float v = sB[r * kS + u];
        sqacc = fmaf(v, v, sqacc);
      }
  }
  // the four slices' tiles, summed in a fixed order: (s0 + s2) + (s1 + s3)
  __syncthreads();
  auto park = [&](float* dst) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      *reinterpret_cast<float4*>(dst + (8 * ti + i) * kS + 8 * tj) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      *reinterpret_cast<float4*>(dst + (8 * ti + i) * kS + 8 * tj + 4) =
          make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
  };
  auto take = [&](const float* src) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 x = *reinterpret_cast<const float4*>(src + (8 * ti + i) * kS + 8 * tj);
      const float4 y = *reinterpret_cast<const float4*>(src + (8 * ti + i) * kS + 8 * tj + 4);
      acc[i][0] += x.x; acc[i][1] += x.y; acc[i][2] += x.z; acc[i][3] += x.w;
      acc[i][4] += y.x; acc[i][5] += y.y; acc[i][6] += y.z; acc[i][7] += y.w;
    }
  };
  if (slice >= 2) park(buf + (slice - 2) * kS * kS);
  if (sq) sq_red[slice][u] = sqacc;
  __syncthreads();
  if (slice < 2) take(buf + slice * kS * kS);
  __syncthreads();
  if (slice == 1) park(buf);
  __syncthreads();
  if (slice == 0) {
    take(buf);
    float* out = pr.part + ((long long)chunk * a.ngroups + g) * kS * kS;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      *reinterpret_cast<float4*>(out + (8 * ti + i) * kS + 8 * tj) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      *reinterpret_cast<float4*>(out + (8 * ti + i) * kS + 8 * tj + 4) =
          make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
  }
  if (sq && t < sg)
    a.sq_part[(long long)chunk * a.W + c0 + t] =
        (sq_red[0][t] + sq_red[2][t]) + (sq_red[1][t] + sq_red[3][t]);
}

// rr_part[chunk][c] = sum over the chunk's rows of R[r][c]^2: CTA (column
// block of 64, chunk), four row slices summed in a fixed order
__global__ void __launch_bounds__(256) k_bcolsq(const float* __restrict__ R, int n, int W,
                                                int rows_per_chunk, float* __restrict__ rr_part) {
  __shared__ float red[4][64];
  const int t = threadIdx.x, c = blockIdx.x * 64 + (t & 63), slice = t >> 6;
  const long long r0 = (long long)blockIdx.y * rows_per_chunk;
  const long long r1 = min((long long)n, r0 + rows_per_chunk);
  float s = 0.f;
  if (c < W)
#pragma unroll 4
    for (long long r = r0 + slice; r < r1; r += 4) {
      const float v = __ldg(R + r * W + c);
      s = fmaf(v, v, s);
    }
  red[slice][t & 63] = s;
  __syncthreads();
  if (slice == 0 && c < W)
    rr_part[(long long)blockIdx.y * W + c] = (red[0][t] + red[2][t]) + (red[1][t] + red[3][t]);
}

// out[e] = sum over chunks of part[chunk][e] in chunk order (FP64); two
// buffers of m elements each (part2/out2 may be null)
__global__ void k_breduce(const float* __restrict__ part, double* __restrict__ out,
                          const float* __restrict__ part2, double* __restrict__ out2, int chunks,
                          long long m) {
  const long long total = part2 ? 2 * m : m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const bool second = e >= m;
    const float* p = second ? part2 : part;
    const long long j = second ? e - m : e;
    double s = 0.0;
#pragma unroll 8
    for (int c = 0; c < chunks; ++c) s += (double)__ldg(p + (long long)c * m + j);
    (second ? out2 : out)[j] = s;
  }
}

// ---------------------------------------------------------------- 64 x 64 algebra (FP64)
// Per group: the Cholesky factor of the unit-scaled matrix and its inverse,
//   D_s S D_s = L L^T,  Li = L^-1 (rows and columns of dropped directions 0),
// so that S^+ = D_s Li^T Li D_s on the kept directions.
struct Factor {
  double Li[kS * kS];
  double dsc[kS];
};

struct FactorSmem {
  double M[kS][kS + 1];
  double Li[kS][kS + 1];
  double dsc[kS];
  int act[kS];
};

// MODE 0: S is the Gram of a direction block; write Tm (float, [g][64][64])
//         with P = T Tm orthonormal on the kept directions: Tm = D_s Li^T.
// MODE 1: S = G = P^T M P; keep the factor for the solves (and open the
//         iteration's count of unconverged groups).
template <int MODE>
__global__ void __launch_bounds__(256) k_bfactor(const double* __restrict__ S_all,
                                                 const int32_t* __restrict__ gdone,
                                                 float* __restrict__ Tm_all,
                                                 Factor* __restrict__ F_all, int32_t* active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FactorSmem& w = *reinterpret_cast<FactorSmem*>(smem_raw);
  const int g = blockIdx.x, t = threadIdx.x;
  if (MODE == 1 && g == 0 && t == 0) *active = 0;
  if (gdone[g]) return;
  const double* S = S_all + (long long)g * kS * kS;
  if (t < kS) {
    const double d = S[t * kS + t];
    w.dsc[t] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
  }
  __syncthreads();
  for (int e = t; e < kS * kS; e += 256) {
    const int i = e >> 6, j = e & 63;
    w.M[i][j] = S[e] * w.dsc[i] * w.dsc[j];
    w.Li[i][j] = 0.0;
  }
  __syncthreads();
  // right-looking Cholesky on the lower triangle
  for (int k = 0; k < kS; ++k) {
    if (t == 0) {
      const double piv = w.M[k][k];
      const bool ok = w.dsc[k] > 0.0 && piv > kDropRel;
      w.act[k] = ok ? 1 : 0;
      w.M[k][k] = ok ? sqrt(piv) : 0.0;
    }
    __syncthreads();
    if (t > k && t < kS) w.M[t][k] = w.act[k] ? w.M[t][k] / w.M[k][k] : 0.0;
    __syncthreads();
    const int m = kS - 1 - k;   // trailing block (k, 64) x (k, 64), lower part
    for (int e = t; e < m * m; e += 256) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (i >= j) w.M[i][j] -= w.M[i][k] * w.M[j][k];
    }
    __syncthreads();
  }
  // Li = L^-1 row by row: Li[i][c] = (delta_ic - sum_{c<=k<i} L[i][k] Li[k][c]) / L[i][i],
  // four threads per c (lanes of one warp) splitting the sum
  const int c = t >> 2, q = t & 3;
  for (int i = 0; i < kS; ++i) {
    double part = 0.0;
    if (c < i)
      for (int k = c + q; k < i; k += 4) part += w.M[i][k] * w.Li[k][c];
    part += __shfl_xor_sync(0xffffffffu, part, 1);
    part += __shfl_xor_sync(0xffffffffu, part, 2);
    if (q == 0 && c <= i)
      w.Li[i][c] = (w.act[i] && w.act[c]) ? ((i == c ? 1.0 : 0.0) - part) / w.M[i][i] : 0.0;
    __syncthreads();
  }
  if (MODE == 0) {
    float* Tm = Tm_all + (long long)g * kS * kS;
    for (int e = t; e < kS * kS; e += 256) {
      const int a = e >> 6, b = e & 63;
      Tm[e] = (float)(w.dsc[a] * w.Li[b][a]);
    }
  } else {
    Factor& f = F_all[g];
    for (int e = t; e < kS * kS; e += 256) f.Li[e] = w.Li[e >> 6][e & 63];
    if (t < kS) f.dsc[t] = w.dsc[t];
  }
}

// out[:, c] = sign * G^+ rhs[:, c], kApplyCols right-hand sides per CTA
// (CTA (g, column block)): z = D_s h, y = Li z, x = D_s Li^T y
__global__ void __launch_bounds__(256) k_bapply(const Factor* __restrict__ F_all,
                                                const double* __restrict__ rhs_all, double sign,
                                                const int32_t* __restrict__ gdone,
                                                float* __restrict__ out_all) {
  __shared__ double Li[kS][kS + 1];
  __shared__ double z[kApplyCols][kS], y[kApplyCols][kS];
  const int g = blockIdx.x, cb = blockIdx.y, t = threadIdx.x;
  if (gdone[g]) return;
  const Factor& f = F_all[g];
  for (int e = t; e < kS * kS; e += 256) Li[e >> 6][e & 63] = f.Li[e];
  const int q = t >> 6, i = t & 63, col = cb * kApplyCols + q;
  const double* rhs = rhs_all + (long long)g * kS * kS;
  z[q][i] = f.dsc[i] * rhs[i * kS + col];
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k <= i; ++k) s += Li[i][k] * z[q][k];
  y[q][i] = s;
  __syncthreads();
  s = 0.0;
  for (int k = i; k < kS; ++k) s += Li[k][i] * y[q][k];
  out_all[(long long)g * kS * kS + i * kS + col] = (float)(sign * f.dsc[i] * s);
}

// a group is done when every column has ||r||^2 <= tol^2 t2 ||r_0||^2 (columns
// past W count as converged); the iteration that ends a group is counted and
// *active counts the groups still open
__global__ void k_bconverge(const double* __restrict__ rr, const double* __restrict__ rr0,
                            const double* __restrict__ t2, int W, double tol2, int32_t* gdone,
                            int32_t* git, int32_t* active) {
  const int g = blockIdx.x, c = threadIdx.x, col = g * kS + c;
  if (gdone[g]) return;
  const bool conv = col >= W || rr[col] <= tol2 * rr0[col] * (t2 ? t2[col] : 1.0);
  const bool all = __syncthreads_and(conv);
  if (c == 0) {
    git[g] += 1;
    if (all)
      gdone[g] = 1;
    else
      atomicAdd(active, 1);
  }
}

// ---------------------------------------------------------------- block products
// out[r][64g + c] = base(r, c) (+/-) sum_k A[r][64g + k] Cm[g][k][c], 128 rows
// per CTA, 128 threads of 8 x 8 tiles:
//   MODE 0: base = out, product added (X += P alpha)
//   MODE 1: base = out, product subtracted (R -= Q alpha)
//   MODE 2: base = scale[r] * Rb[r][.] (T = D^-1 R + P beta)
//   MODE 3: base = 0 (P = T Tm; out may alias A: a CTA stages its rows before writing them)
//   MODE 4: out = scale[r] * A[r][.], no product (the first block D^-1 R)
struct MulArgs {
  const float* A;
  const float* Cm;
  const float* Rb;
  const float* scale;
  float* out;
  int n, W;
  const int32_t* gdone;
};
constexpr size_t kMulSmem = sizeof(float) * (kS * kS + kMulRows * (kS + 1));

template <int MODE>
__global__ void __launch_bounds__(128) k_bmul(const MulArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sC = reinterpret_cast<float*>(smem_raw);   // [64][64]
  float* sA = sC + kS * kS;                          // [128][65]
  const int g = blockIdx.x;
  if (a.gdone[g]) return;
  const int c0 = g * kS, sg = min(kS, a.W - c0);
  const long long r0 = (long long)blockIdx.y * kMulRows;
  const int t = threadIdx.x, rt = t >> 6, u = t & 63, ti = u >> 3, tj = u & 7;
  for (int e = t; e < kMulRows * (kS / 4); e += 128) {
    const int rr = e >> 4, c4 = (e & 15) * 4;
    const long long r = r0 + rr;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < a.n && c4 < sg) v = *reinterpret_cast<const float4*>(a.A + r * a.W + c0 + c4);
    float* d = sA + rr * (kS + 1) + c4;
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
  }
  if (MODE != 4)
    for (int e = t; e < kS * kS / 4; e += 128)
      reinterpret_cast<float4*>(sC)[e] =
          __ldg(reinterpret_cast<const float4*>(a.Cm + (long long)g * kS * kS) + e);
  __syncthreads();
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  const float* arow = sA + (rt * 64 + 8 * ti) * (kS + 1);
  if (MODE != 4) {
#pragma unroll 4
    for (int k = 0; k < kS; ++k) {
      const float4 b0 = *reinterpret_cast<const float4*>(sC + k * kS + 8 * tj);
      const float4 b1 = *reinterpret_cast<const float4*>(sC + k * kS + 8 * tj + 4);
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float av = arow[i * (kS + 1) + k];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av, bv[j], acc[i][j]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long r = r0 + rt * 64 + 8 * ti + i;
    if (r >= a.n) continue;
    const float sr = (MODE == 2 || MODE == 4) ? __ldg(a.scale + r) : 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = 8 * tj + 4 * h;
      if (c >= sg) continue;
      const long long o = r * a.W + c0 + c;
      float4 v = make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2],
                             acc[i][4 * h + 3]);
      if (MODE == 0 || MODE == 1) {
        const float4 b = *reinterpret_cast<const float4*>(a.out + o);
        const float sgn = MODE == 0 ? 1.f : -1.f;
        v = make_float4(fmaf(sgn, v.x, b.x), fmaf(sgn, v.y, b.y), fmaf(sgn, v.z, b.z),
                        fmaf(sgn, v.w, b.w));
      } else if (MODE == 2) {
        const float4 b = __ldg(reinterpret_cast<const float4*>(a.Rb + o));
        v = make_float4(fmaf(sr, b.x, v.x), fmaf(sr, b.y, v.y), fmaf(sr, b.z, v.z),
                        fmaf(sr, b.w, v.w));
      } else if (MODE == 4) {
        const float* s = arow + i * (kS + 1) + c;
        v = make_float4(sr * s[0], sr * s[1], sr * s[2], sr * s[3]);
      }
      *reinterpret_cast<float4*>(a.out + o) = v;
    }
  }
}

__global__ void k_bnarrow(const double* __restrict__ X, long long count, float* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (float)X[e];
}

__global__ void k_bfill_iters(const int32_t* __restrict__ git, int W, int32_t* __restrict__ iters) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < W; c += gridDim.x * blockDim.x)
    iters[c] = git[c / kS];
}

int grid1(long long count) {
  return (int)std::max<long long>(1, std::min<long long>((count + 255) / 256, 152 * 8));
}

}  // namespace

// Workspace of the block solve (one allocation, made on first use and kept by
// the handle for its column count).
struct BcgWs {
  int n = 0, W = 0, ngroups = 0, chunks = 0, rpc = 0;
  float *part = nullptr, *part2 = nullptr, *sq_part = nullptr;
  double *Gm = nullptr, *Hm = nullptr, *rr = nullptr, *rr0 = nullptr;
  Factor* fac = nullptr;
  float *alpha = nullptr, *beta = nullptr, *Tm = nullptr;
  int32_t *gdone = nullptr, *git = nullptr, *zero_done = nullptr, *active = nullptr;
};

namespace {
size_t bcg_carve(BcgWs& b, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = (off + 255) & ~size_t(255);
    char* p = base ? base + off : nullptr;
    off += std::max<size_t>(bytes, 1);
    return p;
  };
  const size_t gm = (size_t)b.ngroups * kS * kS;
  b.part = (float*)take(sizeof(float) * b.chunks * gm);
  b.part2 = (float*)take(sizeof(float) * b.chunks * gm);
  b.sq_part = (float*)take(sizeof(float) * (size_t)b.chunks * b.W);
  b.Gm = (double*)take(sizeof(double) * gm);
  b.Hm = (double*)take(sizeof(double) * gm);
  b.rr = (double*)take(sizeof(double) * b.W);
  b.rr0 = (double*)take(sizeof(double) * b.W);
  b.fac = (Factor*)take(sizeof(Factor) * b.ngroups);
  b.alpha = (float*)take(sizeof(float) * gm);
  b.beta = (float*)take(sizeof(float) * gm);
  b.Tm = (float*)take(sizeof(float) * gm);
  b.gdone = (int32_t*)take(sizeof(int32_t) * b.ngroups);
  b.git = (int32_t*)take(sizeof(int32_t) * b.ngroups);
  b.zero_done = (int32_t*)take(sizeof(int32_t) * b.W);
  b.active = (int32_t*)take(sizeof(int32_t));
  return off;
}

// the kernels above 48 KB of dynamic shared memory (set on every solve: the
// attribute belongs to the current device)
bool bcg_attributes() {
  const int fs = (int)sizeof(FactorSmem), ms = (int)kMulSmem;
  const cudaFuncAttribute attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  return cudaFuncSetAttribute(k_bfactor<0>, attr, fs) == cudaSuccess &&
         cudaFuncSetAttribute(k_bfactor<1>, attr, fs) == cudaSuccess &&
         cudaFuncSetAttribute(k_bmul<0>, attr, ms) == cudaSuccess &&
         cudaFuncSetAttribute(k_bmul<1>, attr, ms) == cudaSuccess &&
         cudaFuncSetAttribute(k_bmul<2>, attr, ms) == cudaSuccess &&
         cudaFuncSetAttribute(k_bmul<3>, attr, ms) == cudaSuccess &&
         cudaFuncSetAttribute(k_bmul<4>, attr, ms) == cudaSuccess;
}

GramArgs gram_args(const BcgWs& b, GramPair p0, GramPair p1, const float* scale_a,
                   float* sq_part) {
  GramArgs a{};
  a.pair[0] = p0;
  a.pair[1] = p1;
  a.npairs = p1.A ? 2 : 1;
  a.scale_a = scale_a;
  a.sq_part = sq_part;
  a.n = b.n;
  a.W = b.W;
  a.ngroups = b.ngroups;
  a.rows_per_chunk = b.rpc;
  a.gdone = b.gdone;
  return a;
}

void gram(const BcgWs& b, GramPair p0, GramPair p1, const float* scale_a, float* sq_part,
          cudaStream_t s) {
  const GramArgs a = gram_args(b, p0, p1, scale_a, sq_part);
  k_bgram<<<dim3(b.ngroups * a.npairs, b.chunks), 256, 0, s>>>(a);
}

template <int MODE>
void bmul(const BcgWs& b, const float* A, const float* Cm, const float* Rb, const float* scale,
          float* out, cudaStream_t s) {
  const dim3 grid(b.ngroups, (unsigned)((b.n + kMulRows - 1) / kMulRows));
  k_bmul<MODE><<<grid, 128, kMulSmem, s>>>(MulArgs{A, Cm, Rb, scale, out, b.n, b.W, b.gdone});
}

// P = orth(T): CholeskyQR twice, the second pass in place on P
void bcg_orth(const BcgWs& b, const float* T, float* P, cudaStream_t s, Launches& L) {
  const long long gm = (long long)b.ngroups * kS * kS;
  const GramPair none{nullptr, nullptr, nullptr};
  const float* src = T;
  for (int pass = 0; pass < 2; ++pass) {
    gram(b, GramPair{src, src, b.part}, none, nullptr, nullptr, s);
    k_breduce<<<grid1(gm), 256, 0, s>>>(b.part, b.Gm, nullptr, nullptr, b.chunks, gm);
    k_bfactor<0><<<b.ngroups, 256, sizeof(FactorSmem), s>>>(b.Gm, b.gdone, b.Tm, nullptr,
                                                            nullptr);
    bmul<3>(b, src, b.Tm, nullptr, nullptr, P, s);
    L.add(4);
    src = P;
  }
}
}  // namespace

void bcg_release(mesh_codec* h) {
  if (h->bcg_mem) cudaFree(h->bcg_mem);
  h->bcg_mem = nullptr;
  delete h->bcg;
  h->bcg = nullptr;
}

int bcg_solve(mesh_codec* h, const CgGeom& geom, const float* inv_d, const float* inv_diag,
              const double* R0, float* X32, float* R32, float* P32, float* T32, float* Q32,
              int32_t* iters, double tol, const double* t2, int max_iters, cudaStream_t s,
              Launches& L) {
  const int n = h->n, W = geom.W;
  if (!bcg_attributes()) return -1;
  if (!h->bcg || h->bcg->W != W || h->bcg->n != n) {
    bcg_release(h);
    BcgWs* b = new BcgWs();
    b->n = n;
    b->W = W;
    b->ngroups = (W + kS - 1) / kS;
    b->rpc = kChunkRows;
    b->chunks = (n + b->rpc - 1) / b->rpc;
    const size_t bytes = bcg_carve(*b, nullptr);
    if (cudaMalloc(&h->bcg_mem, bytes) != cudaSuccess) {
      cudaGetLastError();
      h->bcg_mem = nullptr;
      delete b;
      return -1;
    }
    bcg_carve(*b, (char*)h->bcg_mem);
    h->bcg = b;
    if (cudaMemsetAsync(b->zero_done, 0, sizeof(int32_t) * W, s) != cudaSuccess) return -1;
  }
  const BcgWs& b = *h->bcg;
  const long long nw = (long long)n * W, gm = (long long)b.ngroups * kS * kS;
  const dim3 gapply(b.ngroups, kS / kApplyCols);
  const GramPair none{nullptr, nullptr, nullptr};
  // start: X = 0, R = R0, ||r_0||^2 per column, P = orth(D^-1 R)
  cudaMemsetAsync(X32, 0, sizeof(float) * nw, s);
  cudaMemsetAsync(b.gdone, 0, sizeof(int32_t) * b.ngroups, s);
  cudaMemsetAsync(b.git, 0, sizeof(int32_t) * b.ngroups, s);
  k_bnarrow<<<grid1(nw), 256, 0, s>>>(R0, nw, R32);
  k_bcolsq<<<dim3((W + 63) / 64, b.chunks), 256, 0, s>>>(R32, n, W, b.rpc, b.sq_part);
  k_breduce<<<grid1(W), 256, 0, s>>>(b.sq_part, b.rr0, nullptr, nullptr, b.chunks, W);
  bmul<4>(b, R32, nullptr, nullptr, inv_diag, T32, s);
  L.add(4);
  bcg_orth(b, T32, P32, s, L);
  const double tol2 = tol * tol;
  int it = 0;
  while (it < max_iters) {
    const int m = std::min(kCheck, max_iters - it);
    for (int j = 0; j < m; ++j) {
      // Q = M P (the FP32 operator kernels; their p^T q partials are unused)
      cg4_op(geom, h->row_ptr, h->col_idx, h->deg, inv_d, h->kind, h->is_anchor, P32, T32, Q32,
             b.zero_done, h->cg.partials, s, nullptr);
      // G = P^T Q, H = P^T R; alpha = G^+ H
      gram(b, GramPair{P32, Q32, b.part}, GramPair{P32, R32, b.part2}, nullptr, nullptr, s);
      k_breduce<<<grid1(2 * gm), 256, 0, s>>>(b.part, b.Gm, b.part2, b.Hm, b.chunks, gm);
      k_bfactor<1><<<b.ngroups, 256, sizeof(FactorSmem), s>>>(b.Gm, b.gdone, nullptr, b.fac,
                                                              b.active);
      k_bapply<<<gapply, 256, 0, s>>>(b.fac, b.Hm, 1.0, b.gdone, b.alpha);
      // X += P alpha, R -= Q alpha
      bmul<0>(b, P32, b.alpha, nullptr, nullptr, X32, s);
      bmul<1>(b, Q32, b.alpha, nullptr, nullptr, R32, s);
      // K = (D^-1 Q)^T R and ||r||^2; beta = -G^+ K; convergence
      gram(b, GramPair{Q32, R32, b.part}, none, inv_diag, b.sq_part, s);
      k_breduce<<<grid1(gm), 256, 0, s>>>(b.part, b.Hm, nullptr, nullptr, b.chunks, gm);
      k_breduce<<<grid1(W), 256, 0, s>>>(b.sq_part, b.rr, nullptr, nullptr, b.chunks, W);
      k_bapply<<<gapply, 256, 0, s>>>(b.fac, b.Hm, -1.0, b.gdone, b.beta);
      k_bconverge<<<b.ngroups, kS, 0, s>>>(b.rr, b.rr0, t2, W, tol2, b.gdone, b.git,
                                           b.active);
      // P = orth(D^-1 R + P beta)
      bmul<2>(b, P32, b.beta, R32, inv_diag, T32, s);
      L.add(14);
      bcg_orth(b, T32, P32, s, L);
    }
    it += m;
    if (cudaMemcpyAsync(h->h_active, b.active, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return -1;
    if (*h->h_active == 0) break;
  }
  k_bfill_iters<<<grid1(W), 256, 0, s>>>(b.git, W, iters);
  L.add(1);
  return cudaGetLastError() == cudaSuccess ? it : -1;
}

}  // namespace mc
