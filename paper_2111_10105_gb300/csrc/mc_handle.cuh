// The codec handle (opaque in the C ABI), shared by the translation units
// that enqueue the encoder and decoder.
#pragma once

#include <vector>

#include "mc_internal.cuh"

namespace mc {
struct BcgWs;   // block CG workspace (mc_bcg.cu)
}

// per-decode state carried between the decoder's phases
struct DecodeState {
  bool factored = false;
  bool cached = false;           // factored solve with the kept anchor response G
  bool store = false;            // this decode computes G and may keep it
  bool refine = false;           // FP64 residuals with FP32 CG corrections
  int Wc = 0, single = 0, it = 0;
  mc::CgGeom geom{};
  const void* inv_d = nullptr;
  const void* inv_diag = nullptr;
};

struct mesh_codec {
  mesh_codec_params_t p;
  int n, T, F, k, W, n_c, kind;
  mc::EncodeLayout lay;
  mc::EncodeLayout lay_delta;      // blocks 2..n_b with dictionary differences
  mc::CgGeom geom;
  // device workspace (one allocation)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int32_t *row_ptr, *col_idx, *deg, *anchors, *dec_anchors;
  int32_t* comp;                   // connected-component label per vertex (smallest index)
  uint8_t* is_anchor;
  double *inv_d, *inv_diag;
  float *inv_d32, *inv_diag32;     // FP32 copies for the mixed-precision CG
  double *Q0, *Q, *Zb, *U, *V, *H, *theta, *Wk, *partials, *chg_work, *chg;
  double *G, *Rf;
  double* qr_save;                 // the orthonormalisation's saved input [3][F][k]
  uint32_t* qr_bad;                // its per-coordinate fallback flags
  double *Cf, *qparams;
  double *X, *D, *B, *R, *P, *Tv, *Qv;
  double *Udeq, *Cdeq, *Ahat;
  // mixed modes' factored decode: A^_c U'_c [3][n_c][k] (added to the data
  // columns' right-hand sides at the anchors) and the anchors' residual
  // E_c = A^_c - (A^_c U'_c) U'_c^T [3][n_c][F] (multiplied by G)
  double *AU, *Eanc;
  // blocks variant: the previous block's exact basis (Algorithm 1's start)
  // and the decoder's dequantized previous dictionary [3][F][k]; the direct
  // eigendecomposition of R[1] = A A^T: R and V [3][F][F], eigenvalues [3][F]
  double *Ublk, *Uhat, *Rdir, *Vdir, *thetaF;
  // Anchor response of the factored solve, G = M^-1 P^T ([n][n_c] FP64): it
  // depends only on the connectivity and the anchor set, so the handle keeps
  // the G of its last complete factored decode (own allocation, made on first
  // use) together with that decode's anchors, and later decodes with the
  // same anchors solve only the 3k data columns.  Gcache_anchors holds the
  // anchors of the latest decode (anchors_kept), with or without a G for them:
  // in the automatic solve mode a repeated anchor set switches a frames
  // decode to the factored one, whose G every later decode then reuses.
  double* Gcache = nullptr;
  int32_t* Gcache_anchors = nullptr;
  bool Gcache_valid = false, Gcache_pending = false, anchors_kept = false;
  int32_t* d_match = nullptr;      // device: anchors differing from the kept set
  // refined solve: per column ||B||^2, ||R||^2, converged flag, iterations
  double *ref_bb, *ref_rr, *ref_prev;
  double* ref_t2;                  // per column (inner target / 10^-refine)^2
  int32_t *ref_frozen, *ref_iters;
  // block CG of the refined solve (own allocation, made on first use)
  mc::BcgWs* bcg = nullptr;
  void* bcg_mem = nullptr;
  mc::CgState cg;
  uint32_t* d_status;
  int nnz;
  int max_degree = 0;
  size_t partial_elems;
  // host side
  uint32_t* h_status = nullptr;     // pinned
  int32_t* h_active = nullptr;      // pinned
  uint8_t* h_header = nullptr;      // pinned, 64 bytes
  double* h_chg = nullptr;          // pinned [3]
  // staging for the host-buffer entry points (lazy)
  double* stage_pos = nullptr;
  uint8_t* stage_bits = nullptr;
  cudaStream_t last_stream = nullptr;
  uint64_t launches_create = 0, launches_encode = 0, launches_decode = 0;
  int oi_done[3] = {0, 0, 0};
  double oi_last_change[3] = {0, 0, 0};
  int cg_columns = 0;
  // kernel timing (mesh_codec_set_profiling)
  int prof_every = 0;
  std::vector<cudaEvent_t> prof_events;   // groups of kCgKernels + 1
  size_t prof_used = 0;                    // groups recorded in the current decode
  // whole runs of CG iterations bracketed by one event pair (no per-kernel
  // events inside): the iteration time as the CUDA graph replays it
  std::vector<cudaEvent_t> run_events;     // pairs
  std::vector<int> run_iters;              // iterations inside each recorded pair
  size_t run_used = 0;
  int64_t prof_launches[MESH_CODEC_PROF_KERNELS] = {0};
  double prof_ms[MESH_CODEC_PROF_KERNELS] = {0};
  // mixed precision (precision TF32 / BF16): tensor-core operands and maps
  int lp = -1;                      // 0 tf32 (FP32 storage), 1 bf16; -1 FP64 mode
  int Fp = 0, kp = 0, np = 0;       // frames, rank, vertices padded for TMA boxes
  void *Xlp = nullptr, *XTlp = nullptr, *Dlp = nullptr, *Qtlp = nullptr, *Wtlp = nullptr;
  void *Utlp = nullptr, *Clp = nullptr, *Ulp = nullptr;
  float* tc_part = nullptr;         // split-K partial products
  double* Zfull = nullptr;          // [3][Fp][kp]
  size_t tc_part_elems = 0;
  alignas(64) unsigned char map_X[128], map_Qt[128], map_XT[128], map_Wt[128];
  alignas(64) unsigned char map_D[128], map_Ut[128], map_C[128], map_U[128];
  // decoder's anchor product G A^_c on the tensor cores (own allocation, made
  // on first use): G [n][ncp] and A^_c^T [3][F][ncp], n_c padded to ncp
  void *Glp = nullptr, *Ahlp = nullptr;
  int ncp = 0;
  alignas(64) unsigned char map_G[128], map_Ah[3][128];
  int refine_sweeps = 0;
  // decoder phases, CG geometry autotuning, own stream for the batch entry points
  DecodeState dec;
  mc::CgGeom tuned{};
  int tuned_W = -1, tuned_single = -1;
  cudaStream_t own = nullptr;
  cudaStream_t cap = nullptr;              // capture stream for the CG chunk graph
  // kCgChunk CG iterations [0], and kCgChunk - 1 after a timed one [1]
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  int graph_W[2] = {-1, -1}, graph_single[2] = {-1, -1}, graph_rpb[2] = {-1, -1};
  cudaEvent_t ev_fork = nullptr, ev_done = nullptr, ev_chunk = nullptr;
};

namespace mc {
// the handle's orthonormalisation workspace, split-K over `splits`
inline QrWork qr_work(mesh_codec* h, int splits) {
  return QrWork{h->G, h->Rf, h->partials, h->qr_save, h->qr_bad, splits, h->p.seed};
}
// mixed-precision helpers (mc_mixed.cu)
void mixed_dims(mesh_codec* h);
size_t mixed_carve(mesh_codec* h, char* base, size_t off);
bool mixed_init(mesh_codec* h, cudaStream_t s);
void mixed_oi_sweeps(mesh_codec* h, int sweeps, cudaStream_t s, Launches& L);
void mixed_project(mesh_codec* h, cudaStream_t s, Launches& L);
void mixed_backproject(mesh_codec* h, cudaStream_t s, Launches& L);
bool mixed_finish(mesh_codec* h, const double* Y, long long y_ld, const double* G, long long g_ld,
                  const double* A, bool data_product, cudaStream_t s, Launches& L);
// Block CG (mc_bcg.cu): M D = R0 (R0 FP64 [n][W]) for every column to
// ||r||^2 <= tol^2 t2[col] ||r_0||^2 (t2 null: 1), over groups of 64 columns; D into X32 (FP32), the
// iterations of each column's group into iters.  R32, P32, T32, Q32 are FP32
// [n][W] scratch.  Returns the iterations run, or -1 on a CUDA error.
int bcg_solve(mesh_codec* h, const CgGeom& geom, const float* inv_d, const float* inv_diag,
              const double* R0, float* X32, float* R32, float* P32, float* T32, float* Q32,
              int32_t* iters, double tol, const double* t2, int max_iters, cudaStream_t s,
              Launches& L);
void bcg_release(mesh_codec* h);
}  // namespace mc
