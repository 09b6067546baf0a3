// Dense FP64 kernels of the encoder: the tall-skinny products of orthogonal
// iterations (Algorithm 1 applied as R Q = A (A^T Q), Eq. 7, never forming R),
// the projection of Eq. 9 and the decoder's back-projection (Eq. 11-12), the
// thin QR by shifted CholeskyQR3, and the Rayleigh-Ritz eigen-decomposition
// that orders the retained eigen-trajectories (Eq. 5, Eq. 10).
//
// GB300 executes binary64 at about 2 FMA per SM per clock (no FP64 tensor
// path), so these kernels are bounded by the FP64 pipe: every product is
// spread over all SMs (split-K with a deterministic, fixed-order reduction
// for the long n-sums) and reductions are never left to a single CTA.
#include <algorithm>
#include <math.h>

#include "mc_internal.cuh"

namespace mc {

// ------------------------------------------------------------------ DGEMM
static constexpr int BM = 64, BN = 32, BK = 16, NT = 128;

__global__ void __launch_bounds__(NT) k_dgemm(int M, int N, int K, int batch, int splits,
                                              int kchunk, Strided A, Strided B, StridedOut C,
                                              double* __restrict__ partials) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 8, ty = tid / 8;  // 8 x 16 threads, 4 x 4 outputs each
  const int b = blockIdx.z % batch, split = blockIdx.z / batch;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = split * kchunk, ke = min(K, kb + kchunk);
  const double* Ap = A.p + (long long)b * A.sb;
  const double* Bp = B.p + (long long)b * B.sb;
  const bool a_kfast = (A.s1 == 1), b_nfast = (B.s1 == 1);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / NT; ++q) {
      int e = tid + q * NT;
      int mm, kk;
      if (a_kfast) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < ke) ? Ap[(long long)m * A.s0 + (long long)k * A.s1] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < (BN * BK) / NT; ++q) {
      int e = tid + q * NT;
      int nn, kk;
      if (b_nfast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      int nc = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (nc < N && k < ke) ? Bp[(long long)k * B.s0 + (long long)nc * B.s1] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int nc = n0 + tx * 4 + j;
      if (nc >= N) continue;
      if (splits == 1) {
        double* cp = C.p + (long long)b * C.sb + (long long)m * C.s0 + (long long)nc * C.s1;
        *cp = C.accumulate ? *cp + acc[i][j] : acc[i][j];
      } else {
        partials[(((long long)split * batch + b) * M + m) * N + nc] = acc[i][j];
      }
    }
  }
}

__global__ void k_reduce_partials(int M, int N, int batch, int splits,
                                  const double* __restrict__ partials, StridedOut C) {
  long long total = (long long)batch * M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += partials[(long long)z * total + e];
    long long b = e / ((long long)M * N), r = e % ((long long)M * N);
    long long m = r / N, nc = r % N;
    double* cp = C.p + b * C.sb + m * C.s0 + nc * C.s1;
    *cp = C.accumulate ? *cp + s : s;
  }
}

void dgemm(int M, int N, int K, int batch, Strided A, Strided B, StridedOut C, int splits,
           double* partials, cudaStream_t s, Launches& L) {
  if (splits < 1) splits = 1;
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  splits = (K + kchunk - 1) / kchunk;
  if (splits < 1) splits = 1;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch * splits);
  k_dgemm<<<grid, NT, 0, s>>>(M, N, K, batch, splits, kchunk, A, B, C, partials);
  L.add(1);
  if (splits > 1) {
    long long total = (long long)batch * M * N;
    int g = (int)std::min<long long>((total + 255) / 256, 152 * 8);
    k_reduce_partials<<<g, 256, 0, s>>>(M, N, batch, splits, partials, C);
    L.add(1);
  }
}

// ------------------------------------------------------------ start basis
// Z_c[f][j] = uniform[-1,1) from splitmix64 output f*k + j of
// seed ^ (kBasisSalt + c): top 53 bits times 2^-53, times 2, minus 1 (exact).
__global__ void k_start_basis(double* Z, int F, int k, uint64_t seed) {
  long long per = (long long)F * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 3 * per;
       e += (long long)gridDim.x * blockDim.x) {
    int c = (int)(e / per);
    long long i = e % per;
    uint64_t u = splitmix64_at(seed ^ (kBasisSalt + (uint64_t)c), (uint64_t)i) >> 11;
    Z[e] = (double)u * 0x1.0p-53 * 2.0 - 1.0;
  }
}

void gen_start_basis(double* Z, int F, int k, uint64_t seed, cudaStream_t s, Launches& L) {
  long long total = 3LL * F * k;
  int g = (int)std::min<long long>((total + 255) / 256, 1024);
  k_start_basis<<<g, 256, 0, s>>>(Z, F, k, seed);
  L.add(1);
}

// ------------------------------------------------------------ CholeskyQR3
// Pass 0 factors G + sI with the shift s = 11 (F k + k (k+1)) u ||Z||_F^2
// (Fukaya, Kannan, Nakatsukasa, Zhang, Yamamoto, "Shifted Cholesky QR for
// computing the QR factorization of ill-conditioned matrices", SIAM J. Sci.
// Comput. 2020; ||Z||_F^2 >= ||Z||_2^2 keeps the shift safe), passes 1-2 are
// plain CholeskyQR (CholeskyQR2).  Each pass: G = Z^T Z (split-K DGEMM),
// R = chol(G) upper triangular with positive diagonal (one CTA per
// coordinate), Z <- Z R^-1 (rows in parallel).  The product of the three R
// factors has a positive diagonal, so the result is the unique thin-QR Q.
// A non-positive pivot marks the coordinate in bad[c] (the fallback below
// then recomputes its Q) and leaves R = I, so the pass keeps Z unchanged.
__global__ void __launch_bounds__(1024) k_cholesky(const double* __restrict__ G,
                                                   double* __restrict__ R, int k, int F,
                                                   int shifted, uint32_t* bad) {
  extern __shared__ double A[];  // k x k
  const int c = blockIdx.x;
  const double* Gc = G + (long long)c * k * k;
  double* Rc = R + (long long)c * k * k;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) A[e] = Gc[e];
  __syncthreads();
  if (shifted) {
    __shared__ double sh;
    if (threadIdx.x == 0) {
      double tr = 0.0;
      for (int i = 0; i < k; ++i) tr += A[i * k + i];
      sh = 11.0 * ((double)F * k + (double)k * (k + 1)) * 0x1.0p-53 * tr;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) A[i * k + i] += sh;
    __syncthreads();
  }
  __shared__ int bad_pivot;
  if (threadIdx.x == 0) bad_pivot = 0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    double piv = A[j * k + j];
    if (!(piv > 0.0)) {
      if (threadIdx.x == 0) bad_pivot = 1;
      break;
    }
    double rjj = sqrt(piv);
    double inv = 1.0 / rjj;
    __syncthreads();
    // row j of R
    for (int i = j + threadIdx.x; i < k; i += blockDim.x) A[j * k + i] = (i == j) ? rjj : A[j * k + i] * inv;
    __syncthreads();
    // trailing update A[p][q] -= R[j][p] R[j][q], p, q > j (upper part)
    int m = k - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      int p = j + 1 + e / m, q = j + 1 + e % m;
      if (q >= p) A[p * k + q] -= A[j * k + p] * A[j * k + q];
    }
    __syncthreads();
  }
  __syncthreads();
  if (bad_pivot) {
    if (threadIdx.x == 0) bad[c] = 1;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) Rc[e] = (e / k == e % k) ? 1.0 : 0.0;
    return;
  }
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    int p = e / k, q = e % k;
    Rc[e] = (q >= p) ? A[e] : 0.0;
  }
}

// Z[c] rows: q_j = (z_j - sum_{l<j} q_l R_lj) / R_jj.
__global__ void __launch_bounds__(64) k_trsm_rows(double* __restrict__ Z,
                                                  const double* __restrict__ R, int F, int k) {
  extern __shared__ double Rs[];  // k x k
  const int c = blockIdx.y;
  const double* Rc = R + (long long)c * k * k;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Rs[e] = Rc[e];
  __syncthreads();
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  double* z = Z + ((long long)c * F + f) * k;
  double q[MESH_CODEC_MAX_RANK];
#pragma unroll 1
  for (int j = 0; j < k; ++j) {
    double v = z[j];
    for (int l = 0; l < j; ++l) v = fma(-q[l], Rs[l * k + j], v);
    q[j] = v / Rs[j * k + j];
  }
#pragma unroll 1
  for (int j = 0; j < k; ++j) z[j] = q[j];
}

// bad[c] |= Q_c^T Q_c differs from I by more than 1e-10 anywhere (or is not
// finite): CholeskyQR3 kept every pivot positive but Z was too ill-conditioned
// for it (condition number near 1 / unit roundoff).
__global__ void k_orth_check(const double* __restrict__ G, int k, uint32_t* bad) {
  const int c = blockIdx.x;
  const double* Gc = G + (long long)c * k * k;
  int off = 0;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const double d = Gc[e] - ((e / k == e % k) ? 1.0 : 0.0);
    if (!(fabs(d) <= 1e-10)) off = 1;
  }
  if (__syncthreads_or(off) && threadIdx.x == 0) bad[c] = 1;
}

// Fallback thin QR for the coordinates flagged in bad[]: one CTA per
// coordinate recomputes Q from the saved Z by classical Gram-Schmidt with
// reorthogonalisation (a second pass, and a third while a pass still removes
// more than half the norm: Giraud, Langou, Rozloznik, "The loss of
// orthogonality in the Gram-Schmidt orthogonalization process", Comput.
// Math. Appl. 2005).  A column left with at most 1e-9 of its norm is
// numerically dependent on the earlier ones and is replaced, in this order,
// by the fill column j (the previous iterate, which keeps a completed basis
// stable from sweep to sweep) and by seeded uniform vectors (splitmix64 of
// seed ^ (kCompleteSalt + c), element (attempt * k + j) * F + f).  Full-rank
// columns give the thin-QR Q with a positive diagonal of R, as CholeskyQR3.
constexpr int kQrThreads = 256;

__device__ double qr_block_sum(double x, double* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = x;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kQrThreads / 32; ++w) s += red[w];
  return s;
}

__global__ void __launch_bounds__(kQrThreads) k_qr_robust(double* __restrict__ Z,
                                                          const double* __restrict__ save,
                                                          const double* __restrict__ fill, int F,
                                                          int k, const uint32_t* __restrict__ bad,
                                                          uint64_t seed, uint32_t* status) {
  const int c = blockIdx.x;
  if (!bad[c]) return;
  extern __shared__ double sm[];
  double* v = sm;                                    // [F] the column being built
  double* r = v + F;                                 // [k] projection coefficients
  double* red = r + MESH_CODEC_MAX_RANK;             // [(threads / 32) * k] partial sums
  double* Q = Z + (long long)c * F * k;
  const double* S = save + (long long)c * F * k;
  const double* Fl = fill ? fill + (long long)c * F * k : nullptr;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  for (int j = 0; j < k; ++j) {
    bool done = false;
    for (int attempt = 0; attempt < 5 && !done; ++attempt) {
      for (int f = tid; f < F; f += kQrThreads) {
        double x;
        if (attempt == 0) {
          x = S[(long long)f * k + j];
        } else if (attempt == 1 && Fl) {
          x = Fl[(long long)f * k + j];
        } else {
          const uint64_t u = splitmix64_at(seed ^ (kCompleteSalt + (uint64_t)c),
                                           ((uint64_t)attempt * k + j) * F + f) >> 11;
          x = (double)u * 0x1.0p-53 * 2.0 - 1.0;
        }
        v[f] = x;
      }
      __syncthreads();
      double part = 0.0;
      for (int f = tid; f < F; f += kQrThreads) part += v[f] * v[f];
      const double n0 = sqrt(qr_block_sum(part, red));
      if (!(n0 > 0.0) || !isfinite(n0)) continue;
      double nv = n0;
      for (int pass = 0; pass < 3 && j > 0; ++pass) {
        // r_i = q_i . v for i < j: per-thread partials, then warp and block sums
        double acc[MESH_CODEC_MAX_RANK];
#pragma unroll
        for (int i = 0; i < MESH_CODEC_MAX_RANK; ++i) acc[i] = 0.0;
        for (int f = tid; f < F; f += kQrThreads) {
          const double vf = v[f];
          const double* qrow = Q + (long long)f * k;
#pragma unroll
          for (int i = 0; i < MESH_CODEC_MAX_RANK; ++i)
            if (i < j) acc[i] = fma(qrow[i], vf, acc[i]);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < MESH_CODEC_MAX_RANK; ++i) {
          if (i < j) {
            double x = acc[i];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) red[warp * MESH_CODEC_MAX_RANK + i] = x;
          }
        }
        __syncthreads();
        for (int i = tid; i < j; i += kQrThreads) {
          double x = 0.0;
          for (int w = 0; w < kQrThreads / 32; ++w) x += red[w * MESH_CODEC_MAX_RANK + i];
          r[i] = x;
        }
        __syncthreads();
        part = 0.0;
        for (int f = tid; f < F; f += kQrThreads) {
          const double* qrow = Q + (long long)f * k;
          double x = v[f];
          for (int i = 0; i < j; ++i) x = fma(-r[i], qrow[i], x);
          v[f] = x;
          part += x * x;
        }
        const double nn = sqrt(qr_block_sum(part, red));
        const bool enough = !(nn < 0.5 * nv);
        nv = nn;
        if (enough) break;
      }
      if (nv > 1e-9 * n0 && isfinite(nv)) {
        const double inv = 1.0 / nv;
        for (int f = tid; f < F; f += kQrThreads) Q[(long long)f * k + j] = v[f] * inv;
        done = true;
      }
      __syncthreads();
    }
    if (!done) {
      if (tid == 0) atomicOr(status, ST_CHOL_BREAKDOWN);
      return;
    }
  }
}

__global__ void k_flag_bad(const uint32_t* bad, uint32_t* status) {
  if (threadIdx.x < 3 && bad[threadIdx.x]) atomicOr(status, ST_CHOL_BREAKDOWN);
}

void cholqr3(double* Z, int F, int k, const QrWork& w, const double* fill, uint32_t* status,
             cudaStream_t s, Launches& L) {
  cudaMemcpyAsync(w.save, Z, sizeof(double) * 3 * F * k, cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(w.bad, 0, sizeof(uint32_t) * 3, s);
  Strided A{Z, 1, k, (long long)F * k};
  Strided B{Z, k, 1, (long long)F * k};
  StridedOut C{w.G, k, 1, (long long)k * k};
  for (int pass = 0; pass < 3; ++pass) {
    // G_c = Z_c^T Z_c : (k x F)(F x k)
    dgemm(k, k, F, 3, A, B, C, w.splits, w.partials, s, L);
    k_cholesky<<<3, 256, sizeof(double) * k * k, s>>>(w.G, w.R, k, F, pass == 0, w.bad);
    dim3 g((F + 63) / 64, 3);
    k_trsm_rows<<<g, 64, sizeof(double) * k * k, s>>>(Z, w.R, F, k);
    L.add(2);
  }
  // orthogonality of the result, then the fallback where it failed
  dgemm(k, k, F, 3, A, B, C, w.splits, w.partials, s, L);
  k_orth_check<<<3, 256, 0, s>>>(w.G, k, w.bad);
  const size_t smem = sizeof(double) * (F + MESH_CODEC_MAX_RANK +
                                        (kQrThreads / 32) * MESH_CODEC_MAX_RANK);
  if (smem > 227 * 1024) {
    // the column does not fit in shared memory (F above ~28,000 frames): a
    // flagged coordinate is reported instead of repaired
    k_flag_bad<<<1, 32, 0, s>>>(w.bad, status);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_qr_robust, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_qr_robust<<<3, kQrThreads, smem, s>>>(Z, w.save, fill, F, k, w.bad, w.seed, status);
  }
  L.add(2);
}

// ||Q_new - Q_old (Q_old^T Q_new)||_F per coordinate; P = Q_old (Q_old^T Q_new)
// is formed by two DGEMMs, then this kernel reduces the squared difference.
__global__ void k_change(const double* __restrict__ Qn, const double* __restrict__ P, int F,
                         int k, double* change) {
  __shared__ double sh[256];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (long long e = threadIdx.x; e < (long long)F * k; e += blockDim.x) {
    double d = Qn[(long long)c * F * k + e] - P[(long long)c * F * k + e];
    acc = fma(d, d, acc);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) change[c] = sqrt(sh[0]);
}

void oi_change(const double* Qold, const double* Qnew, int F, int k, double* work,
               double* change, cudaStream_t s, Launches& L) {
  double* Mk = work;                       // [3][k][k]
  double* P = work + 3LL * k * k;          // [3][F][k]
  dgemm(k, k, F, 3, Strided{Qold, 1, k, (long long)F * k}, Strided{Qnew, k, 1, (long long)F * k},
        StridedOut{Mk, k, 1, (long long)k * k}, 1, nullptr, s, L);
  dgemm(F, k, k, 3, Strided{Qold, k, 1, (long long)F * k}, Strided{Mk, k, 1, (long long)k * k},
        StridedOut{P, k, 1, (long long)F * k}, 1, nullptr, s, L);
  k_change<<<3, 256, 0, s>>>(Qnew, P, F, k, change);
  L.add(1);
}

// ------------------------------------------------------------ Jacobi eig
// Cyclic two-sided Jacobi on the symmetric k x k Rayleigh quotient H (one CTA
// per coordinate), parallel round-robin ordering: every round rotates k'/2
// disjoint pairs (k' = k rounded up to even, the padding index has a zero
// row).  Rotation as in Golub & Van Loan, Matrix Computations, Alg. 8.5.2
// (sym.schur2).  A pair is skipped when |H_pq| <= 2^-54 sqrt(|H_pp H_qq|)
// (or below the smallest normal).  Stops after a sweep without rotations.
// Output: eigenvalues descending (ties: lower index first) and the matching
// eigenvector columns.
__global__ void __launch_bounds__(256) k_jacobi(const double* __restrict__ Hin,
                                                double* __restrict__ Vout,
                                                double* __restrict__ theta, int k) {
  extern __shared__ double smem[];
  const int kp = (k + 1) & ~1;
  double* H = smem;              // kp x kp
  double* V = H + kp * kp;       // kp x kp
  double* cs = V + kp * kp;      // kp/2 x 2
  int* arr = (int*)(cs + kp);    // kp
  int* pr = arr + kp;            // kp/2 x 2
  __shared__ int rotated;
  const int c = blockIdx.x;
  const double* Hc = Hin + (long long)c * k * k;
  for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) {
    int p = e / kp, q = e % kp;
    H[e] = (p < k && q < k) ? 0.5 * (Hc[p * k + q] + Hc[q * k + p]) : 0.0;
    V[e] = (p == q) ? 1.0 : 0.0;
  }
  for (int i = threadIdx.x; i < kp; i += blockDim.x) arr[i] = i;
  __syncthreads();
  const int half = kp / 2;
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < kp - 1; ++round) {
      for (int i = threadIdx.x; i < half; i += blockDim.x) {
        int p = arr[i], q = arr[kp - 1 - i];
        if (p > q) { int t = p; p = q; q = t; }
        pr[2 * i] = p;
        pr[2 * i + 1] = q;
        double apq = H[p * kp + q], app = H[p * kp + p], aqq = H[q * kp + q];
        double cc = 1.0, ss = 0.0;
        if (fabs(apq) > 2.2250738585072014e-308 &&
            fabs(apq) > 0x1.0p-54 * sqrt(fabs(app) * fabs(aqq))) {
          double tau = (aqq - app) / (2.0 * apq);
          double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          cc = 1.0 / sqrt(1.0 + t * t);
          ss = t * cc;
          rotated = 1;
        }
        cs[2 * i] = cc;
        cs[2 * i + 1] = ss;
      }
      __syncthreads();
      // rows: H <- J^T H
      for (int e = threadIdx.x; e < half * kp; e += blockDim.x) {
        int i = e / kp, col = e % kp;
        int p = pr[2 * i], q = pr[2 * i + 1];
        double cc = cs[2 * i], ss = cs[2 * i + 1];
        if (ss == 0.0) continue;
        double hp = H[p * kp + col], hq = H[q * kp + col];
        H[p * kp + col] = cc * hp - ss * hq;
        H[q * kp + col] = ss * hp + cc * hq;
      }
      __syncthreads();
      // columns: H <- H J, V <- V J
      for (int e = threadIdx.x; e < half * kp; e += blockDim.x) {
        int i = e / kp, row = e % kp;
        int p = pr[2 * i], q = pr[2 * i + 1];
        double cc = cs[2 * i], ss = cs[2 * i + 1];
        if (ss == 0.0) continue;
        double hp = H[row * kp + p], hq = H[row * kp + q];
        H[row * kp + p] = cc * hp - ss * hq;
        H[row * kp + q] = ss * hp + cc * hq;
        double vp = V[row * kp + p], vq = V[row * kp + q];
        V[row * kp + p] = cc * vp - ss * vq;
        V[row * kp + q] = ss * vp + cc * vq;
      }
      __syncthreads();
      // rotate the tournament (element 0 fixed)
      if (threadIdx.x == 0) {
        int last = arr[kp - 1];
        for (int i = kp - 1; i > 1; --i) arr[i] = arr[i - 1];
        arr[1] = last;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  // sort: rank of each eigenvalue among the first k (descending, ties by index)
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double tj = H[j * kp + j];
    int rank = 0;
    for (int i = 0; i < k; ++i) {
      double ti = H[i * kp + i];
      rank += (ti > tj) || (ti == tj && i < j);
    }
    theta[(long long)c * k + rank] = tj;
    for (int r = 0; r < k; ++r) Vout[(long long)c * k * k + r * k + rank] = V[r * kp + j];
  }
}

void jacobi_eig(const double* H, double* V, double* theta, int k, cudaStream_t s, Launches& L) {
  int kp = (k + 1) & ~1;
  size_t sm = sizeof(double) * (2 * kp * kp + kp) + sizeof(int) * (2 * kp);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_jacobi<<<3, 256, sm, s>>>(H, V, theta, k);
  L.add(1);
}

// Sign of each eigenvector (left open by the paper): make sum_f (f+1) u_f > 0,
// or, when |sum| < 1e-12 ||u||_1 F, the entry of largest magnitude positive
// (lowest index on ties).
__global__ void k_sign_rule(double* U, int F, int k) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * k) return;
  int c = t / k, j = t % k;
  double* u = U + (long long)c * F * k;
  double s = 0.0, l1 = 0.0, best = -1.0, at = 0.0;
  for (int f = 0; f < F; ++f) {
    double v = u[(long long)f * k + j];
    s = fma((double)(f + 1), v, s);
    l1 += fabs(v);
    if (fabs(v) > best) { best = fabs(v); at = v; }
  }
  if (fabs(s) < 1e-12 * l1 * F) s = at;
  if (s < 0.0)
    for (int f = 0; f < F; ++f) u[(long long)f * k + j] = -u[(long long)f * k + j];
}

void sign_rule(double* U, int F, int k, cudaStream_t s, Launches& L) {
  k_sign_rule<<<(3 * k + 63) / 64, 64, 0, s>>>(U, F, k);
  L.add(1);
}

}  // namespace mc
