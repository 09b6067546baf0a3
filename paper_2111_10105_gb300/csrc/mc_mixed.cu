// Mixed-precision forms of the encoder's dense products (TF32 or BF16
// operands on tcgen05 tensor cores, FP32 accumulation; FP64 everywhere the
// codec decides something):
//   orthogonal-iteration sweeps  W_c = A_c^T Q_c,  Z_c = A_c W_c  (Algorithm 1,
//     Eq. 7) as two tensor-core GEMMs per sweep, the K = n reduction split
//     over CTAs and summed in FP64; the QR of Z stays FP64 (CholeskyQR3);
//   then FP64 refinement sweeps and the FP64 Rayleigh-Ritz of the FP64 path;
//   the projection C_c = U_c^T delta_c^T (Eq. 9) and the decoder's
//   back-projection delta~_c = (U_c' C_c')^T (Eq. 11) as tensor-core GEMMs;
//   the factored decoder's X_c = Y_c U_c'^T + G E_c (Eq. 12 reassociated:
//   A^_c = (A^_c U'_c) U'_c^T + E_c, the first part solved with the data
//   columns) as two tensor-core GEMMs, the second adding onto the first's
//   FP64 result.
//
// Operand layouts (all K-major for the TN kernel, padded so that every TMA
// box starts on a 16-byte boundary; padding is zero):
//   Xlp, Dlp [n][3][Fp]   positions / delta coordinates (vertex rows, frames)
//   XTlp     [3][Fp][np]  positions, frame rows (the K = n operand of A_c W)
//   Qtlp     [3][kp][Fp]  Q_c^T;   Wtlp [3][kp][np]  W_c^T
//   Utlp     [3][kp][Fp]  U_c^T;   Clp [3][n][kp] C_c'^T (or Y_c);  Ulp [3][F][kp] U_c'
//   Glp      [n][ncp]     G;       Ahlp [3][F][ncp] A^_c^T   (ncp = n_c padded to 64)
#include <algorithm>

#include "mc_handle.cuh"

namespace mc {

static long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

// element bytes of the low-precision operands
static int lp_bytes(const mesh_codec* h) { return h->lp == 0 ? 4 : 2; }

size_t mixed_carve(mesh_codec* h, char* base, size_t off) {
  if (h->lp < 0) return off;
  auto take = [&](size_t bytes) -> char* {
    off = (off + 1023) & ~size_t(1023);
    char* p = base ? base + off : nullptr;
    off += std::max<size_t>(bytes, 1);
    return p;
  };
  const size_t eb = lp_bytes(h), n = h->n, F = h->F;
  const size_t Fp = h->Fp, kp = h->kp, np = h->np;
  h->Xlp = take(eb * n * 3 * Fp);
  h->XTlp = take(eb * 3 * Fp * np);
  h->Dlp = take(eb * n * 3 * Fp);
  h->Qtlp = take(eb * 3 * kp * Fp);
  h->Wtlp = take(eb * 3 * kp * np);
  h->Utlp = take(eb * 3 * kp * Fp);
  h->Clp = take(eb * 3 * n * kp);
  h->Ulp = take(eb * 3 * F * kp);
  h->tc_part = (float*)take(sizeof(float) * h->tc_part_elems);
  h->Zfull = (double*)take(sizeof(double) * 3 * Fp * kp);
  return off;
}

// K splits of the A_c W product: enough CTAs to cover the SMs twice
static int z_splits(const mesh_codec* h) {
  const int atom = h->lp == 0 ? 32 : 64;
  const long long chunks = (h->np + atom - 1) / atom;
  const long long tiles = 3LL * ((h->Fp + 127) / 128);
  long long s = std::max<long long>(1, (152 * 2) / tiles);
  return (int)std::min<long long>(s, chunks);
}

void mixed_dims(mesh_codec* h) {
  const int p = h->p.precision;
  h->lp = p == MC_PRECISION_TF32 ? 0 : (p == MC_PRECISION_BF16 ? 1 : -1);
  if (h->lp < 0) return;
  h->Fp = (int)round_up(h->F, 64);
  h->kp = (int)round_up(h->k, 16);
  h->np = (int)round_up(h->n, 64);
  h->tc_part_elems = (size_t)z_splits(h) * 3 * h->Fp * h->kp;
}

// zero the padding once and build the TMA descriptors of the fixed buffers
bool mixed_init(mesh_codec* h, cudaStream_t s) {
  if (h->lp < 0) return true;
  const int eb = lp_bytes(h);
  const long long n = h->n, F = h->F, Fp = h->Fp, kp = h->kp, np = h->np;
  cudaMemsetAsync(h->XTlp, 0, (size_t)eb * 3 * Fp * np, s);
  cudaMemsetAsync(h->Qtlp, 0, (size_t)eb * 3 * kp * Fp, s);
  cudaMemsetAsync(h->Wtlp, 0, (size_t)eb * 3 * kp * np, s);
  cudaMemsetAsync(h->Utlp, 0, (size_t)eb * 3 * kp * Fp, s);
  bool ok = true;
  ok &= tc_operand_map(h->map_X, h->Xlp, eb, Fp, n, 3, 3 * Fp, Fp, 128);
  ok &= tc_operand_map(h->map_Qt, h->Qtlp, eb, Fp, kp, 3, Fp, kp * Fp, tc_bn((int)kp));
  ok &= tc_operand_map(h->map_XT, h->XTlp, eb, np, Fp, 3, np, Fp * np, 128);
  ok &= tc_operand_map(h->map_Wt, h->Wtlp, eb, np, kp, 3, np, kp * np, tc_bn((int)kp));
  ok &= tc_operand_map(h->map_D, h->Dlp, eb, Fp, n, 3, 3 * Fp, Fp, 128);
  ok &= tc_operand_map(h->map_Ut, h->Utlp, eb, Fp, kp, 3, Fp, kp * Fp, tc_bn((int)kp));
  ok &= tc_operand_map(h->map_C, h->Clp, eb, kp, n, 3, kp, n * kp, 128);
  ok &= tc_operand_map(h->map_U, h->Ulp, eb, kp, F, 3, kp, F * kp, tc_bn((int)F));
  return ok;
}

// Z [3][F][k] = crop of Zfull [3][Fp][kp]
__global__ void k_crop(const double* __restrict__ Zf, int F, int k, int Fp, int kp,
                       double* __restrict__ Z) {
  const long long total = 3LL * F * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long c = e / ((long long)F * k), r = e % ((long long)F * k);
    long long f = r / k, j = r % k;
    Z[e] = Zf[(c * Fp + f) * kp + j];
  }
}

static void pack_Qt(mesh_codec* h, const double* Q, void* dst, cudaStream_t s, Launches& L) {
  // dst[c][j][f] = Q_c[f][j]
  pack_operand_f64(Q, (long long)h->F * h->k, 1, h->k, 3, h->k, h->F, h->Fp, h->Fp,
                   (long long)h->kp * h->Fp, h->lp, dst, s, L);
}

// tensor-core orthogonal-iteration sweeps from h->Q (FP64 in, FP64 out)
void mixed_oi_sweeps(mesh_codec* h, int sweeps, cudaStream_t s, Launches& L) {
  const long long n = h->n, F = h->F, k = h->k, W = h->W;
  const long long Fp = h->Fp, kp = h->kp, np = h->np;
  const int out_lp = h->lp == 0 ? 1 : 2;
  // positions as the two low-precision operands
  pack_operand_f64(h->X, F, W, 1, 3, n, F, Fp, 3 * Fp, Fp, h->lp, h->Xlp, s, L);
  pack_operand_f64(h->X, F, 1, W, 3, F, n, n, np, Fp * np, h->lp, h->XTlp, s, L);
  pack_Qt(h, h->Q, h->Qtlp, s, L);
  const int sg = std::max(1, std::min(16, (int)(F / 64)));
  const int zs = z_splits(h);
  for (int t = 0; t < sweeps; ++t) {
    // W_c^T = (A_c^T Q_c)^T : M = n vertices, N = kp, K = Fp
    umma_tn(h->lp, h->map_X, h->map_Qt, (int)n, (int)kp, (int)Fp, 3, 1, h->Wtlp, out_lp, 1, np,
            kp * np, 0, h->d_status, s, L);
    // Z_c = A_c W_c : M = Fp frames, N = kp, K = np vertices, split over K
    int used = umma_tn(h->lp, h->map_XT, h->map_Wt, (int)Fp, (int)kp, (int)np, 3, zs, h->tc_part,
                       0, kp, 1, Fp * kp, 3 * Fp * kp, h->d_status, s, L);
    sum_splits(h->tc_part, used, 3 * Fp * kp, 3 * Fp * kp, h->Zfull, s, L);
    k_crop<<<(int)std::min<long long>((3 * F * k + 255) / 256, 1024), 256, 0, s>>>(
        h->Zfull, (int)F, (int)k, (int)Fp, (int)kp, h->Zb);
    L.add(1);
    cholqr3(h->Zb, (int)F, (int)k, qr_work(h, sg), h->Q, h->d_status, s, L);
    std::swap(h->Q, h->Zb);
    if (t + 1 < sweeps) pack_Qt(h, h->Q, h->Qtlp, s, L);
  }
}

// C_c = U_c^T delta_c^T on the tensor cores, written as FP64 [3][k][n]
void mixed_project(mesh_codec* h, cudaStream_t s, Launches& L) {
  const long long n = h->n, F = h->F, k = h->k, W = h->W, Fp = h->Fp, kp = h->kp;
  pack_operand_f64(h->D, F, W, 1, 3, n, F, Fp, 3 * Fp, Fp, h->lp, h->Dlp, s, L);
  pack_Qt(h, h->U, h->Utlp, s, L);
  umma_tn(h->lp, h->map_D, h->map_Ut, (int)n, (int)k, (int)Fp, 3, 1, h->Cf, 3, 1, n, k * n, 0,
          h->d_status, s, L);
}

// delta~_c = (U_c' C_c')^T on the tensor cores into D [n][3F] (FP64)
void mixed_backproject(mesh_codec* h, cudaStream_t s, Launches& L) {
  const long long n = h->n, F = h->F, k = h->k, W = h->W, kp = h->kp;
  // Clp[c][i][r] = C'_c[r][i],  Ulp[c][f][r] = U'_c[f][r]
  pack_operand_f64(h->Cdeq, k * n, 1, n, 3, n, k, kp, kp, n * kp, h->lp, h->Clp, s, L);
  pack_operand_f64(h->Udeq, F * k, k, 1, 3, F, k, kp, kp, F * kp, h->lp, h->Ulp, s, L);
  umma_tn(h->lp, h->map_C, h->map_U, (int)n, (int)F, (int)kp, 3, 1, h->D, 3, W, 1, F, 0,
          h->d_status, s, L);
}

// X_c = Y_c U_c'^T + G A_c into D [n][3F] (FP64) on the tensor cores: Y the
// 3k data columns of the solve (Y_c at Y + c k, row pitch y_ld), G the anchor
// response [n][n_c] (row pitch g_ld), A [3][n_c][F] the anchors' term; without
// data_product only G A_c is added onto D.  False when the anchor operands
// cannot be allocated or described; nothing is enqueued then.
bool mixed_finish(mesh_codec* h, const double* Y, long long y_ld, const double* G, long long g_ld,
                  const double* A, bool data_product, cudaStream_t s, Launches& L) {
  const long long n = h->n, F = h->F, k = h->k, W = h->W, kp = h->kp, n_c = h->n_c;
  const int eb = lp_bytes(h);
  if (n_c > 0 && !h->Glp) {
    const long long ncp = round_up(n_c, 64);
    void *g = nullptr, *a = nullptr;
    if (cudaMalloc(&g, (size_t)eb * n * ncp) != cudaSuccess ||
        cudaMalloc(&a, (size_t)eb * 3 * F * ncp) != cudaSuccess) {
      cudaGetLastError();
      if (g) cudaFree(g);
      return false;
    }
    bool ok = tc_operand_map(h->map_G, g, eb, ncp, n, 1, ncp, n * ncp, 128);
    for (int c = 0; c < 3; ++c)
      ok &= tc_operand_map(h->map_Ah[c], (char*)a + (size_t)eb * c * F * ncp, eb, ncp, F, 1, ncp,
                           F * ncp, tc_bn((int)F));
    if (!ok) {
      cudaFree(g);
      cudaFree(a);
      return false;
    }
    h->Glp = g;
    h->Ahlp = a;
    h->ncp = (int)ncp;
  }
  if (data_product) {
    // Clp[c][i][r] = Y_c[i][r],  Ulp[c][f][r] = U'_c[f][r]
    pack_operand_f64(Y, k, y_ld, 1, 3, n, k, kp, kp, n * kp, h->lp, h->Clp, s, L);
    pack_operand_f64(h->Udeq, F * k, k, 1, 3, F, k, kp, kp, F * kp, h->lp, h->Ulp, s, L);
    umma_tn(h->lp, h->map_C, h->map_U, (int)n, (int)F, (int)kp, 3, 1, h->D, 3, W, 1, F, 0,
            h->d_status, s, L);
  }
  if (n_c == 0) return true;
  const long long ncp = h->ncp;
  // Glp[i][a] = G[i][a],  Ahlp[c][f][a] = A_c[a][f]
  pack_operand_f64(G, 0, g_ld, 1, 1, n, n_c, ncp, ncp, n * ncp, h->lp, h->Glp, s, L);
  pack_operand_f64(A, n_c * F, 1, F, 3, F, n_c, ncp, ncp, F * ncp, h->lp, h->Ahlp, s, L);
  for (int c = 0; c < 3; ++c)
    umma_tn(h->lp, h->map_G, h->map_Ah[c], (int)n, (int)F, (int)ncp, 1, 1, h->D + c * F, 4, W,
            1, 0, 0, h->d_status, s, L);
  return true;
}

}  // namespace mc
