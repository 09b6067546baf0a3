// Learned warm start: a 3-layer perceptron (n_in -> H -> H -> n_out, ReLU)
// with BF16 weights and FP32 accumulation, trained on the GPU by its own
// forward, backward and Adam kernels; plus the kernel that assembles the
// per vertex-frame features it reads (previous segment's reconstruction,
// displacement of the nearest anchor, change of the decoded delta
// coordinates).  Its prediction is only a first iterate of the decoder's CG
// (mesh_codec_decode_ex): the solution of Eq. 12 does not depend on it.
//
// Parameters are one flat FP32 master array [W1 (H x n_in), b1, W2 (H x H),
// b2, W3 (n_out x H), b3] with a BF16 copy used by every product; the Adam
// moments are FP32.  Loss: mean squared error over all outputs.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "mc_internal.cuh"

using namespace mc;

struct mesh_codec_mlp {
  int nin, nh, nout;
  size_t count;
  size_t oW1, ob1, oW2, ob2, oW3, ob3;
  float *master = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
  __nv_bfloat16* wbf = nullptr;
  // activations, grown to the largest batch seen
  float *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *dY = nullptr, *dH2 = nullptr, *dH1 = nullptr;
  size_t cap_n = 0;
  float* part = nullptr;
  size_t cap_part = 0;
  double* loss_dev = nullptr;
  double* loss_host = nullptr;   // pinned
  long long step = 0;
  int fp32_weights = 0;   // check mode: products use the float32 master weights
  // input standardisation x' = (x - mu) * inv_sigma (identity until fitted)
  float *mu = nullptr, *inv_sigma = nullptr, *Xn = nullptr;
  double* stat_part = nullptr;
  // tensor-core inference (mesh_codec_mlp_infer): W2 widened to float32 (exact
  // from bfloat16, the TF32 operand), the TMA descriptors of H1 and W2, and
  // the GEMM's status word (made on first use)
  float* W2f = nullptr;
  uint32_t *tc_status = nullptr, *tc_status_host = nullptr;
  alignas(64) unsigned char map_H1[128], map_W2[128];
  uint64_t tc_launches = 0;
};

namespace {

// rows per chunk of an inference call (activations: 4 x n_hidden floats per row)
constexpr long long kForwardChunk = 1LL << 22;

// ---------------------------------------------------------------- SIMT GEMM
// C(m, n) = sum_k A(m, k) B(k, n) in FP32, A and B float or bf16, strided;
// split-K partials summed in a fixed order by k_sum_partials_f.
constexpr int TM = 64, TN = 64, TK = 16;

template <typename T>
__device__ __forceinline__ float ldf(const T* p) { return (float)*p; }
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const TA* __restrict__ A,
                                               long long as0, long long as1,
                                               const TB* __restrict__ B, long long bs0,
                                               long long bs1, float* __restrict__ out,
                                               long long cs0, long long cs1, int kchunk) {
  __shared__ float As[TK][TM + 1];
  __shared__ float Bs[TK][TN + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  // row tiles on x (up to 2^31 - 1 of them), column tiles on y (n <= 4096)
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += TK) {
    for (int e = tid; e < TM * TK; e += 256) {
      int mm, kk;
      if (as1 == 1) { kk = e % TK; mm = e / TK; } else { mm = e % TM; kk = e / TM; }
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < ke) ? ldf(A + (long long)m * as0 + (long long)k * as1) : 0.f;
    }
    for (int e = tid; e < TN * TK; e += 256) {
      int nn, kk;
      if (bs1 == 1) { nn = e % TN; kk = e / TN; } else { kk = e % TK; nn = e / TK; }
      const int nc = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (nc < N && k < ke) ? ldf(B + (long long)k * bs0 + (long long)nc * bs1) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* o = out + (long long)blockIdx.z * M * N;   // partial plane (or C itself, z = 0)
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nc = n0 + tx * 4 + j;
      if (nc < N) {
        if (gridDim.z == 1) o[(long long)m * cs0 + (long long)nc * cs1] = acc[i][j];
        else o[(long long)m * N + nc] = acc[i][j];
      }
    }
  }
}

__global__ void k_sum_partials_f(const float* __restrict__ part, int splits, int M, int N,
                                 float* __restrict__ C, long long cs0, long long cs1) {
  const long long total = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[(long long)z * total + e];
    C[(e / N) * cs0 + (e % N) * cs1] = s;
  }
}

template <typename TA, typename TB>
void sgemm(mesh_codec_mlp* m, int M, int N, int K, const TA* A, long long as0, long long as1,
           const TB* B, long long bs0, long long bs1, float* C, long long cs0, long long cs1,
           cudaStream_t s) {
  int splits = 1;
  const long long tiles = (long long)((M + TM - 1) / TM) * ((N + TN - 1) / TN);
  if (tiles < 152 && K > 4096) {
    splits = (int)std::min<long long>(std::max<long long>(1, 304 / tiles), K / 1024);
    while ((size_t)splits * M * N > m->cap_part && splits > 1) --splits;
  }
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + TK - 1) / TK * TK;
  splits = (K + kchunk - 1) / kchunk;
  dim3 grid((M + TM - 1) / TM, (N + TN - 1) / TN, splits);
  k_sgemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, as0, as1, B, bs0, bs1,
                                       splits == 1 ? C : m->part, cs0, cs1, kchunk);
  if (splits > 1) {
    const long long total = (long long)M * N;
    k_sum_partials_f<<<(int)std::min<long long>((total + 255) / 256, 1024), 256, 0, s>>>(
        m->part, splits, M, N, C, cs0, cs1);
  }
}

// Z[i][j] += b[j], then ReLU (relu = 1) in place
__global__ void k_bias_act(float* Z, const float* __restrict__ b, long long N, int C, int relu) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * C;
       e += (long long)gridDim.x * blockDim.x) {
    float v = Z[e] + b[e % C];
    Z[e] = relu ? fmaxf(v, 0.f) : v;
  }
}

// dY = 2 (Y - T) / (N C); per-block partial sums of (Y - T)^2 in FP64
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, long long total,
                      float scale, float* __restrict__ dY, double* __restrict__ loss_part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const float d = Y[e] - T[e];
    dY[e] = 2.f * d * scale;
    acc += (double)d * (double)d;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = sh[0];
}

__global__ void k_loss_final(const double* __restrict__ part, int nb, double scale, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    out[0] = s * scale;
  }
}

// dH *= (H > 0)
__global__ void k_relu_mask(float* dH, const float* __restrict__ H, long long total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    if (!(H[e] > 0.f)) dH[e] = 0.f;
}

// g[j] = sum_i D[i][j], fixed order: a thread per column, partial over a row
// range per block.y, then k_sum_partials_f over the blocks
__global__ void k_colsum_part(const float* __restrict__ D, long long N, int C, long long rows,
                              float* __restrict__ part) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= C) return;
  const long long r0 = (long long)blockIdx.y * rows, r1 = std::min<long long>(N, r0 + rows);
  float s = 0.f;
  for (long long i = r0; i < r1; ++i) s += D[i * C + j];
  part[(long long)blockIdx.y * C + j] = s;
}

void colsum(mesh_codec_mlp* m, const float* D, long long N, int C, float* g, cudaStream_t s) {
  int blocks = (int)std::min<long long>(std::max<long long>(1, N / 256),
                                        (long long)(m->cap_part / std::max(C, 1)));
  blocks = std::max(1, std::min(blocks, 1024));
  const long long rows = (N + blocks - 1) / blocks;
  dim3 grid((C + 127) / 128, blocks);
  k_colsum_part<<<grid, 128, 0, s>>>(D, N, C, rows, m->part);
  k_sum_partials_f<<<(C + 255) / 256, 256, 0, s>>>(m->part, blocks, 1, C, g, 0, 1);
}

// Adam (Kingma & Ba 2015) on the FP32 master copy, then the BF16 copy
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, __nv_bfloat16* __restrict__ wb, long long count,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const float gr = g[e];
    const float a = b1 * m1[e] + (1.f - b1) * gr;
    const float v = b2 * m2[e] + (1.f - b2) * gr * gr;
    m1[e] = a;
    m2[e] = v;
    const float wn = w[e] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    w[e] = wn;
    wb[e] = __float2bfloat16_rn(wn);
  }
}

__global__ void k_fill_f(float* p, int count, float v) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) p[i] = v;
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb,
                          long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    wb[e] = __float2bfloat16_rn(w[e]);
}

__global__ void k_from_bf16(const __nv_bfloat16* __restrict__ wb, float* __restrict__ out,
                            long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = __bfloat162float(wb[e]);
}

// He-uniform weights from splitmix64 (bound sqrt(6 / fan_in)); the output
// layer is scaled by 0.1 so that the first prediction is close to zero;
// biases zero
__global__ void k_init_params(float* w, long long count, uint64_t seed, long long oW1,
                              long long ob1, long long oW2, long long ob2, long long oW3,
                              long long ob3, int nin, int nh) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const double u = (double)(splitmix64_at(seed, (uint64_t)e) >> 11) * 0x1.0p-53 * 2.0 - 1.0;
    float v = 0.f;
    if (e < ob1) v = (float)(u * sqrt(6.0 / nin));
    else if (e >= oW2 && e < ob2) v = (float)(u * sqrt(6.0 / nh));
    else if (e >= oW3 && e < ob3) v = (float)(0.1 * u * sqrt(6.0 / nh));
    w[e] = v;
  }
}

int grid_for(long long work) {
  return (int)std::max<long long>(1, std::min<long long>((work + 255) / 256, 152 * 16));
}

mesh_codec_status_t ensure_batch(mesh_codec_mlp* m, size_t N) {
  if (N <= m->cap_n) return MC_OK;
  float** bufs[7] = {&m->H1, &m->H2, &m->Y, &m->dY, &m->dH2, &m->dH1, &m->Xn};
  const size_t widths[7] = {(size_t)m->nh, (size_t)m->nh, (size_t)m->nout, (size_t)m->nout,
                            (size_t)m->nh, (size_t)m->nh, (size_t)m->nin};
  for (int i = 0; i < 7; ++i) {
    if (*bufs[i]) cudaFree(*bufs[i]);
    *bufs[i] = nullptr;
    if (cudaMalloc(bufs[i], sizeof(float) * N * widths[i]) != cudaSuccess) {
      m->cap_n = 0;
      return MC_E_OOM;
    }
  }
  m->cap_n = N;
  return MC_OK;
}

// Xn = (X - mu) * inv_sigma, columns of a row-major [N][C] array
__global__ void k_standardize(const float* __restrict__ X, long long N, int C,
                              const float* __restrict__ mu, const float* __restrict__ is,
                              float* __restrict__ Xn) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * C;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % C);
    Xn[e] = (X[e] - mu[j]) * is[j];
  }
}

// per-column sums of x and x^2 in float64 over a row range per block.y
__global__ void k_colstats_part(const float* __restrict__ X, long long N, int C, long long rows,
                                double* __restrict__ part) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= C) return;
  const long long r0 = (long long)blockIdx.y * rows;
  const long long r1 = r0 + rows < N ? r0 + rows : N;
  double s1 = 0.0, s2 = 0.0;
  for (long long i = r0; i < r1; ++i) {
    const double x = X[i * C + j];
    s1 += x;
    s2 += x * x;
  }
  part[2 * ((long long)blockIdx.y * C + j)] = s1;
  part[2 * ((long long)blockIdx.y * C + j) + 1] = s2;
}

// mean and 1 / standard deviation (population); a column whose standard
// deviation is below 1e-12 (relative to its mean's magnitude or absolute)
// keeps inv_sigma = 1
__global__ void k_colstats_final(const double* __restrict__ part, int blocks, int C, long long N,
                                 float* __restrict__ mu, float* __restrict__ is) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= C) return;
  double s1 = 0.0, s2 = 0.0;
  for (int b = 0; b < blocks; ++b) {
    s1 += part[2 * ((long long)b * C + j)];
    s2 += part[2 * ((long long)b * C + j) + 1];
  }
  const double m = s1 / (double)N;
  const double var = fmax(s2 / (double)N - m * m, 0.0);
  const double sd = sqrt(var);
  mu[j] = (float)m;
  is[j] = sd > 1e-12 * fmax(1.0, fabs(m)) ? (float)(1.0 / sd) : 1.f;
}

// WT: __nv_bfloat16 (the bfloat16 copy) or float (the master weights, check mode)
template <typename WT>
void forward_w(mesh_codec_mlp* m, const WT* w, const float* X, long long N, float* Y,
               cudaStream_t s) {
  const int nin = m->nin, nh = m->nh, nout = m->nout;
  const float* p = m->master;
  // Xn = standardised X; H1 = relu(Xn W1^T + b1), H2 = relu(H1 W2^T + b2), Y = H2 W3^T + b3
  k_standardize<<<grid_for(N * nin), 256, 0, s>>>(X, N, nin, m->mu, m->inv_sigma, m->Xn);
  sgemm(m, (int)N, nh, nin, (const float*)m->Xn, nin, 1, w + m->oW1, 1, nin, m->H1, nh, 1, s);
  k_bias_act<<<grid_for(N * nh), 256, 0, s>>>(m->H1, p + m->ob1, N, nh, 1);
  sgemm(m, (int)N, nh, nh, m->H1, nh, 1, w + m->oW2, 1, nh, m->H2, nh, 1, s);
  k_bias_act<<<grid_for(N * nh), 256, 0, s>>>(m->H2, p + m->ob2, N, nh, 1);
  sgemm(m, (int)N, nout, nh, m->H2, nh, 1, w + m->oW3, 1, nh, Y, nout, 1, s);
  k_bias_act<<<grid_for(N * nout), 256, 0, s>>>(Y, p + m->ob3, N, nout, 0);
}

// loss into loss_dev[0] and the gradients of all parameters into m->grad
template <typename WT>
void backward_w(mesh_codec_mlp* m, const WT* w, const float* X, const float* T, long long N,
                cudaStream_t s) {
  const int nin = m->nin, nh = m->nh, nout = m->nout;
  float* g = m->grad;
  const long long tot = N * nout;
  const int nb = 256;
  k_mse<<<nb, 256, 0, s>>>(m->Y, T, tot, 1.f / (float)tot, m->dY, m->loss_dev + 1);
  k_loss_final<<<1, 32, 0, s>>>(m->loss_dev + 1, nb, 1.0 / (double)tot, m->loss_dev);
  // layer 3: dW3 = dY^T H2, db3 = colsum(dY), dH2 = (dY W3) .* (H2 > 0)
  sgemm(m, nout, nh, (int)N, m->dY, 1, nout, m->H2, nh, 1, g + m->oW3, nh, 1, s);
  colsum(m, m->dY, N, nout, g + m->ob3, s);
  sgemm(m, (int)N, nh, nout, m->dY, nout, 1, w + m->oW3, nh, 1, m->dH2, nh, 1, s);
  k_relu_mask<<<grid_for(N * nh), 256, 0, s>>>(m->dH2, m->H2, N * nh);
  // layer 2
  sgemm(m, nh, nh, (int)N, m->dH2, 1, nh, m->H1, nh, 1, g + m->oW2, nh, 1, s);
  colsum(m, m->dH2, N, nh, g + m->ob2, s);
  sgemm(m, (int)N, nh, nh, m->dH2, nh, 1, w + m->oW2, nh, 1, m->dH1, nh, 1, s);
  k_relu_mask<<<grid_for(N * nh), 256, 0, s>>>(m->dH1, m->H1, N * nh);
  // layer 1 (on the standardised inputs the forward pass left in Xn)
  sgemm(m, nh, nin, (int)N, m->dH1, 1, nh, (const float*)m->Xn, nin, 1, g + m->oW1, nin, 1, s);
  colsum(m, m->dH1, N, nh, g + m->ob1, s);
}

void forward(mesh_codec_mlp* m, const float* X, long long N, float* Y, cudaStream_t s) {
  if (m->fp32_weights) forward_w(m, (const float*)m->master, X, N, Y, s);
  else forward_w(m, (const __nv_bfloat16*)m->wbf, X, N, Y, s);
}

void backward(mesh_codec_mlp* m, const float* X, const float* T, long long N, cudaStream_t s) {
  if (m->fp32_weights) backward_w(m, (const float*)m->master, X, T, N, s);
  else backward_w(m, (const __nv_bfloat16*)m->wbf, X, T, N, s);
}

// forward_w with the hidden-to-hidden product H1 W2^T (nh x nh of the
// n_in*nh + nh*nh + nh*n_out multiply-adds per row) on the tensor cores:
// kind::tf32, the bfloat16 weights exact in TF32, the float32 activations
// rounded to TF32 by the MMA, float32 accumulation in TMEM.  False when the
// operands cannot be described for TMA (nothing enqueued then).
bool infer_tc(mesh_codec_mlp* m, const float* X, long long N, float* Y, cudaStream_t s) {
  const int nin = m->nin, nh = m->nh, nout = m->nout;
  const float* p = m->master;
  const __nv_bfloat16* w = m->wbf;
  if (!tc_operand_map(m->map_H1, m->H1, 4, nh, N, 1, nh, N * nh, 128)) return false;
  Launches L{&m->tc_launches};
  k_standardize<<<grid_for(N * nin), 256, 0, s>>>(X, N, nin, m->mu, m->inv_sigma, m->Xn);
  sgemm(m, (int)N, nh, nin, (const float*)m->Xn, nin, 1, w + m->oW1, 1, nin, m->H1, nh, 1, s);
  k_bias_act<<<grid_for(N * nh), 256, 0, s>>>(m->H1, p + m->ob1, N, nh, 1);
  umma_tn(0, m->map_H1, m->map_W2, (int)N, nh, nh, 1, 1, m->H2, 0, nh, 1, 0, 0, m->tc_status, s,
          L);
  k_bias_act<<<grid_for(N * nh), 256, 0, s>>>(m->H2, p + m->ob2, N, nh, 1);
  sgemm(m, (int)N, nout, nh, m->H2, nh, 1, w + m->oW3, 1, nh, Y, nout, 1, s);
  k_bias_act<<<grid_for(N * nout), 256, 0, s>>>(Y, p + m->ob3, N, nout, 0);
  return true;
}

// ---------------------------------------------------------------- features
// kWarmFeatures float32 per sample e = f*n + v (frame f of the current
// segment, vertex v), for the kWarmAnchors nearest anchors a_j = nearest[v][j]:
//   [4j .. 4j+2] a_cur(a_j, f) - x_last(anchors[a_j])   anchor displacement
//   [4j + 3]     dist[v][j]                             rest-pose distance
//   [12 .. 14]   (delta_cur(v, f) - delta_prev(v, F-1)) * dscale
//   [15]         (f + 1) / F
// and, when x_cur != null, target[e] = x_cur(v, f) - x_last(v).
// x_last [n][3] (the previous segment's last frame); x_cur [F][n][3];
// a_cur [3][n_c][F]; delta_cur, delta_prev vertex-major [n][3F].
constexpr int kWarmAnchors = 3, kWarmFeatures = 16;

__global__ void k_features(int n, int F, int n_c, const double* __restrict__ x_last,
                           const double* __restrict__ a_cur, const int32_t* __restrict__ anchors,
                           const int32_t* __restrict__ nearest, const float* __restrict__ dist,
                           const double* __restrict__ d_cur, const double* __restrict__ d_prev,
                           float dscale, const double* __restrict__ x_cur, float* __restrict__ feat,
                           float* __restrict__ target) {
  const long long total = (long long)n * F;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long f = e / n, v = e % n;
    float* o = feat + e * kWarmFeatures;
    for (int j = 0; j < kWarmAnchors; ++j) {
      const int an = nearest[v * kWarmAnchors + j];
      const long long av = anchors[an];
      for (int c = 0; c < 3; ++c)
        o[4 * j + c] = (float)(a_cur[((long long)c * n_c + an) * F + f] - x_last[av * 3 + c]);
      o[4 * j + 3] = dist[v * kWarmAnchors + j];
    }
    for (int c = 0; c < 3; ++c) {
      const long long row = v * 3LL * F + (long long)c * F;
      o[12 + c] = (float)((d_cur[row + f] - d_prev[row + F - 1]) * dscale);
      if (target) target[e * 3 + c] = (float)(x_cur[(f * n + v) * 3 + c] - x_last[v * 3 + c]);
    }
    o[15] = (float)(f + 1) / (float)F;
  }
}

// X0(f, v, c) = x_last(v, c) + pred[f*n + v][c] (pred may be null)
__global__ void k_compose(int n, int F, const double* __restrict__ x_last,
                          const float* __restrict__ pred, double* __restrict__ x0) {
  const long long total = (long long)n * F * 3;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long vc = e % (3LL * n);
    x0[e] = x_last[vc] + (pred ? (double)pred[e] : 0.0);
  }
}

// out[i] = X[r_i] (rows of `width` floats), r_i = splitmix64(seed, i) mod N
__global__ void k_sample_rows(const float* __restrict__ X, int width, long long N, uint64_t seed,
                              long long count, float* __restrict__ out) {
  const long long total = count * width;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / width;
    const long long r = (long long)(splitmix64_at(seed, (uint64_t)i) % (uint64_t)N);
    out[e] = X[r * width + e % width];
  }
}

// basis head: row (c, f) of U_prev [3][F][k] -> features [U_prev(c, f, :), (f + 1) / F]
// (k + 1 floats); target U_cur - U_prev (k floats)
__global__ void k_basis_features(int F, int k, const double* __restrict__ U_prev,
                                 const double* __restrict__ U_cur, float* __restrict__ feat,
                                 float* __restrict__ target) {
  const long long rows = 3LL * F;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * (k + 1);
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / (k + 1);
    const int j = (int)(e % (k + 1));
    if (j < k) {
      feat[e] = (float)U_prev[r * k + j];
      if (target) target[r * k + j] = (float)(U_cur[r * k + j] - U_prev[r * k + j]);
    } else {
      feat[e] = (float)((r % F) + 1) / (float)F;
    }
  }
}

// q0 = U_prev + pred ([3][F][k])
__global__ void k_basis_compose(long long total, const double* __restrict__ U_prev,
                                const float* __restrict__ pred, double* __restrict__ q0) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    q0[e] = U_prev[e] + (pred ? (double)pred[e] : 0.0);
}

// the kWarmAnchors nearest anchors (Euclidean, rest pose [n][3]) of every
// vertex, nearest first, ties by lower anchor index; fewer anchors than
// kWarmAnchors repeat the last one found
__global__ void k_nearest_anchor(int n, int n_c, const double* __restrict__ rest,
                                 const int32_t* __restrict__ anchors, int32_t* __restrict__ nearest,
                                 float* __restrict__ dist) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    double bd[kWarmAnchors];
    int bi[kWarmAnchors];
    for (int j = 0; j < kWarmAnchors; ++j) { bd[j] = 1e300; bi[j] = -1; }
    for (int a = 0; a < n_c; ++a) {
      const long long u = anchors[a];
      double d2 = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double t = rest[v * 3 + c] - rest[u * 3 + c];
        d2 = __dadd_rn(d2, __dmul_rn(t, t));   // no contraction: sum of rounded squares
      }
      // insertion into the sorted list; equal distances keep the earlier index
      int j = kWarmAnchors;
      while (j > 0 && d2 < bd[j - 1]) --j;
      if (j < kWarmAnchors) {
        for (int t = kWarmAnchors - 1; t > j; --t) { bd[t] = bd[t - 1]; bi[t] = bi[t - 1]; }
        bd[j] = d2;
        bi[j] = a;
      }
    }
    for (int j = 0; j < kWarmAnchors; ++j) {
      const int src = bi[j] >= 0 ? j : (j > 0 ? j - 1 : 0);
      if (bi[j] < 0) { bi[j] = bi[src]; bd[j] = bd[src]; }
      nearest[v * kWarmAnchors + j] = bi[j];
      dist[v * kWarmAnchors + j] = (float)sqrt(bd[j]);
    }
  }
}

}  // namespace

extern "C" {

mesh_codec_status_t mesh_codec_mlp_create(int n_in, int n_hidden, int n_out, uint64_t seed,
                                          mesh_codec_mlp_t** out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 4096 || n_hidden > 4096 ||
      n_out > 4096)
    return MC_E_INVALID_ARG;
  *out = nullptr;
  mesh_codec_mlp* m = new (std::nothrow) mesh_codec_mlp();
  if (!m) return MC_E_OOM;
  m->nin = n_in;
  m->nh = n_hidden;
  m->nout = n_out;
  m->oW1 = 0;
  m->ob1 = m->oW1 + (size_t)n_hidden * n_in;
  m->oW2 = m->ob1 + n_hidden;
  m->ob2 = m->oW2 + (size_t)n_hidden * n_hidden;
  m->oW3 = m->ob2 + n_hidden;
  m->ob3 = m->oW3 + (size_t)n_out * n_hidden;
  m->count = m->ob3 + n_out;
  m->cap_part = std::max<size_t>((size_t)8 * n_hidden * std::max(n_hidden, n_in), 1 << 20);
  bool ok = cudaMalloc(&m->master, sizeof(float) * m->count) == cudaSuccess &&
            cudaMalloc(&m->grad, sizeof(float) * m->count) == cudaSuccess &&
            cudaMalloc(&m->m1, sizeof(float) * m->count) == cudaSuccess &&
            cudaMalloc(&m->m2, sizeof(float) * m->count) == cudaSuccess &&
            cudaMalloc(&m->wbf, sizeof(__nv_bfloat16) * m->count) == cudaSuccess &&
            cudaMalloc(&m->part, sizeof(float) * m->cap_part) == cudaSuccess &&
            cudaMalloc(&m->loss_dev, sizeof(double) * 260) == cudaSuccess &&
            cudaMalloc(&m->mu, sizeof(float) * n_in) == cudaSuccess &&
            cudaMalloc(&m->inv_sigma, sizeof(float) * n_in) == cudaSuccess &&
            cudaMalloc(&m->stat_part, sizeof(double) * 2 * 1024 * n_in) == cudaSuccess &&
            cudaMallocHost(&m->loss_host, sizeof(double)) == cudaSuccess;
  if (!ok) {
    mesh_codec_mlp_destroy(m);
    return MC_E_OOM;
  }
  k_init_params<<<grid_for((long long)m->count), 256>>>(m->master, (long long)m->count, seed,
                                                        m->oW1, m->ob1, m->oW2, m->ob2, m->oW3,
                                                        m->ob3, n_in, n_hidden);
  k_to_bf16<<<grid_for((long long)m->count), 256>>>(m->master, m->wbf, (long long)m->count);
  cudaMemset(m->m1, 0, sizeof(float) * m->count);
  cudaMemset(m->m2, 0, sizeof(float) * m->count);
  cudaMemset(m->mu, 0, sizeof(float) * n_in);
  k_fill_f<<<1, 256>>>(m->inv_sigma, n_in, 1.f);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    mesh_codec_mlp_destroy(m);
    return MC_E_CUDA;
  }
  *out = m;
  return MC_OK;
}

size_t mesh_codec_mlp_param_count(const mesh_codec_mlp_t* m) { return m ? m->count : 0; }

mesh_codec_status_t mesh_codec_mlp_get_params(const mesh_codec_mlp_t* m, int which, float* dst,
                                              void* stream) {
  if (!m || !dst || which < 0 || which > 2) return MC_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (which == 0)
    cudaMemcpyAsync(dst, m->master, sizeof(float) * m->count, cudaMemcpyDeviceToDevice, s);
  else if (which == 1)
    k_from_bf16<<<grid_for((long long)m->count), 256, 0, s>>>(m->wbf, dst, (long long)m->count);
  else
    cudaMemcpyAsync(dst, m->grad, sizeof(float) * m->count, cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

mesh_codec_status_t mesh_codec_mlp_set_params(mesh_codec_mlp_t* m, const float* src,
                                              void* stream) {
  if (!m || !src) return MC_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemcpyAsync(m->master, src, sizeof(float) * m->count, cudaMemcpyDeviceToDevice, s);
  k_to_bf16<<<grid_for((long long)m->count), 256, 0, s>>>(m->master, m->wbf, (long long)m->count);
  cudaMemsetAsync(m->m1, 0, sizeof(float) * m->count, s);
  cudaMemsetAsync(m->m2, 0, sizeof(float) * m->count, s);
  m->step = 0;
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

mesh_codec_status_t mesh_codec_mlp_forward(mesh_codec_mlp_t* m, const float* X, long long N,
                                           float* Y, void* stream) {
  if (!m || !X || !Y || N < 1) return MC_E_INVALID_ARG;
  // inference over many rows runs in chunks, so the activations stay small
  const long long chunk = std::min<long long>(N, kForwardChunk);
  mesh_codec_status_t st = ensure_batch(m, (size_t)chunk);
  if (st != MC_OK) return st;
  for (long long r = 0; r < N; r += chunk)
    forward(m, X + r * m->nin, std::min(chunk, N - r), Y + r * m->nout, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

mesh_codec_status_t mesh_codec_mlp_infer(mesh_codec_mlp_t* m, const float* X, long long N,
                                         float* Y, void* stream) {
  if (!m || !X || !Y || N < 1) return MC_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long chunk = std::min<long long>(N, kForwardChunk);
  mesh_codec_status_t st = ensure_batch(m, (size_t)chunk);
  if (st != MC_OK) return st;
  const int nh = m->nh;
  if (!m->W2f) {
    if (cudaMalloc(&m->W2f, sizeof(float) * nh * nh) != cudaSuccess ||
        cudaMalloc(&m->tc_status, sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&m->tc_status_host, sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      return MC_E_OOM;
    }
  }
  if (!tc_operand_map(m->map_W2, m->W2f, 4, nh, nh, 1, nh, (long long)nh * nh, tc_bn(nh)))
    return mesh_codec_mlp_forward(m, X, N, Y, stream);   // FP32-product forward instead
  k_from_bf16<<<grid_for((long long)nh * nh), 256, 0, s>>>(m->wbf + m->oW2, m->W2f,
                                                           (long long)nh * nh);
  cudaMemsetAsync(m->tc_status, 0, sizeof(uint32_t), s);
  for (long long r = 0; r < N; r += chunk) {
    const long long rows = std::min(chunk, N - r);
    if (!infer_tc(m, X + r * m->nin, rows, Y + r * m->nout, s))
      forward(m, X + r * m->nin, rows, Y + r * m->nout, s);
  }
  cudaMemcpyAsync(m->tc_status_host, m->tc_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return MC_E_CUDA;
  if (*m->tc_status_host != 0) return MC_E_CUDA;
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

mesh_codec_status_t mesh_codec_mlp_train_step(mesh_codec_mlp_t* m, const float* X,
                                              const float* T, long long N, float lr,
                                              int update, double* loss, void* stream) {
  if (!m || !X || !T || N < 1 || !(lr >= 0.f)) return MC_E_INVALID_ARG;
  mesh_codec_status_t st = ensure_batch(m, (size_t)N);
  if (st != MC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  forward(m, X, N, m->Y, s);
  backward(m, X, T, N, s);
  if (update) {
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    k_adam<<<grid_for((long long)m->count), 256, 0, s>>>(m->master, m->grad, m->m1, m->m2, m->wbf,
                                                         (long long)m->count, lr, b1, b2, 1e-8f,
                                                         c1, c2);
  }
  if (loss) {
    cudaMemcpyAsync(m->loss_host, m->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return MC_E_CUDA;
    *loss = *m->loss_host;
  }
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

mesh_codec_status_t mesh_codec_mlp_fit_normalizer(mesh_codec_mlp_t* m, const float* X, long long N,
                                                  void* stream) {
  if (!m || !X || N < 1) return MC_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int C = m->nin;
  const int blocks = (int)std::max<long long>(1, std::min<long long>(1024, N / 256));
  const long long rows = (N + blocks - 1) / blocks;
  dim3 grid((C + 127) / 128, blocks);
  k_colstats_part<<<grid, 128, 0, s>>>(X, N, C, rows, m->stat_part);
  k_colstats_final<<<(C + 127) / 128, 128, 0, s>>>(m->stat_part, blocks, C, N, m->mu,
                                                   m->inv_sigma);
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

mesh_codec_status_t mesh_codec_mlp_get_normalizer(const mesh_codec_mlp_t* m, float* mu,
                                                  float* inv_sigma, void* stream) {
  if (!m || !mu || !inv_sigma) return MC_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemcpyAsync(mu, m->mu, sizeof(float) * m->nin, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(inv_sigma, m->inv_sigma, sizeof(float) * m->nin, cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

mesh_codec_status_t mesh_codec_mlp_set_check_mode(mesh_codec_mlp_t* m, int fp32_weights) {
  if (!m || fp32_weights < 0 || fp32_weights > 1) return MC_E_INVALID_ARG;
  m->fp32_weights = fp32_weights;
  return MC_OK;
}

void mesh_codec_mlp_destroy(mesh_codec_mlp_t* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  float* bufs[] = {m->master, m->grad, m->m1, m->m2, m->H1, m->H2, m->Y, m->dY, m->dH2, m->dH1,
                   m->part, m->mu, m->inv_sigma, m->Xn};
  for (float* b : bufs)
    if (b) cudaFree(b);
  if (m->wbf) cudaFree(m->wbf);
  if (m->loss_dev) cudaFree(m->loss_dev);
  if (m->loss_host) cudaFreeHost(m->loss_host);
  if (m->stat_part) cudaFree(m->stat_part);
  if (m->W2f) cudaFree(m->W2f);
  if (m->tc_status) cudaFree(m->tc_status);
  if (m->tc_status_host) cudaFreeHost(m->tc_status_host);
  delete m;
}

mesh_codec_status_t mesh_codec_nearest_anchor(int n, int n_c, const double* rest,
                                              const int32_t* anchors, int32_t* nearest,
                                              float* dist, void* stream) {
  if (n < 1 || n_c < 1 || !rest || !anchors || !nearest || !dist) return MC_E_INVALID_ARG;
  k_nearest_anchor<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, n_c, rest, anchors, nearest,
                                                                  dist);
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

mesh_codec_status_t mesh_codec_warm_features(int n, int F, int n_c, const double* x_last,
                                             const double* a_cur, const int32_t* anchors,
                                             const int32_t* nearest, const float* dist,
                                             const double* delta_cur, const double* delta_prev,
                                             float dscale, const double* x_cur, float* features,
                                             float* target, void* stream) {
  if (n < 1 || F < 1 || n_c < 1 || !x_last || !a_cur || !anchors || !nearest || !dist ||
      !delta_cur || !delta_prev || !features || (x_cur && !target))
    return MC_E_INVALID_ARG;
  k_features<<<grid_for((long long)n * F), 256, 0, (cudaStream_t)stream>>>(
      n, F, n_c, x_last, a_cur, anchors, nearest, dist, delta_cur, delta_prev, dscale, x_cur,
      features, x_cur ? target : nullptr);
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

mesh_codec_status_t mesh_codec_warm_compose(int n, int F, const double* x_last, const float* pred,
                                            double* x0, void* stream) {
  if (n < 1 || F < 1 || !x_last || !x0) return MC_E_INVALID_ARG;
  k_compose<<<grid_for((long long)n * F * 3), 256, 0, (cudaStream_t)stream>>>(n, F, x_last, pred,
                                                                             x0);
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

mesh_codec_status_t mesh_codec_sample_rows(const float* X, int width, long long N, uint64_t seed,
                                           long long count, float* out, void* stream) {
  if (!X || !out || width < 1 || N < 1 || count < 1) return MC_E_INVALID_ARG;
  k_sample_rows<<<grid_for(count * width), 256, 0, (cudaStream_t)stream>>>(X, width, N, seed,
                                                                          count, out);
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

mesh_codec_status_t mesh_codec_basis_features(int F, int k, const double* U_prev,
                                              const double* U_cur, float* features, float* target,
                                              void* stream) {
  if (F < 1 || k < 1 || !U_prev || !features || (U_cur && !target)) return MC_E_INVALID_ARG;
  k_basis_features<<<grid_for(3LL * F * (k + 1)), 256, 0, (cudaStream_t)stream>>>(
      F, k, U_prev, U_cur, features, U_cur ? target : nullptr);
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

mesh_codec_status_t mesh_codec_basis_compose(int F, int k, const double* U_prev, const float* pred,
                                             double* q0, void* stream) {
  if (F < 1 || k < 1 || !U_prev || !q0) return MC_E_INVALID_ARG;
  k_basis_compose<<<grid_for(3LL * F * k), 256, 0, (cudaStream_t)stream>>>(3LL * F * k, U_prev,
                                                                          pred, q0);
  return cudaGetLastError() == cudaSuccess ? MC_OK : MC_E_CUDA;
}

}  // extern "C"
