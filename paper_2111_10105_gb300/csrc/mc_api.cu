// C ABI of the codec (include/mesh_codec.h): handle, workspace and the order
// in which the encoder and decoder enqueue their kernels.
//
// Encoder, per call (Section III, Fig. 1):
//   ingest [F][n][3] -> X [n][3F]; delta = L X (Eq. 3/4, Eq. 8);
//   orthogonal iterations Q <- qr(A_c (A_c^T Q)) (Algorithm 1, Eq. 7) for the
//   three coordinates at once; Rayleigh-Ritz (eigen-order, sign); projection
//   C_c = U_c^T delta_c^T (Eq. 9, first k rows = Eq. 10's truncation);
//   quantize + pack dictionary, coefficients and anchor positions.
// Decoder (Eq. 11-12): unpack; delta~ = (U' C')^T; B = L^T delta~ + P^T a^;
//   Jacobi-CG on (L^T L + P^T P) X = B over all 3F columns; X -> [F][n][3].
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "mc_internal.cuh"

using namespace mc;

#include "mc_handle.cuh"

namespace {

// the blocks variant's first block takes U[1] from the eigendecomposition of
// R[1] = A A^T while its F x F matrix fits the Jacobi eigensolver
constexpr int kDirectMaxFrames = MESH_CODEC_MAX_RANK;

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? (T*)(base + off) : nullptr;
    off += sizeof(T) * std::max<size_t>(count, 1);
    return p;
  }
};

// lay out (or measure, when base == nullptr) the workspace
size_t carve(mesh_codec* h, void* base) {
  Carver c(base);
  const size_t n = h->n, F = h->F, k = h->k, nc = std::max(h->n_c, 1);
  // CG columns, either mode (factored: 3k + n_c, padded to a multiple of 4)
  const size_t W = std::max<size_t>(h->W, (3 * k + h->n_c + 3) / 4 * 4);
  const size_t nnz_max = 6ull * h->T;
  h->row_ptr = c.take<int32_t>(n + 1);
  h->col_idx = c.take<int32_t>(nnz_max);
  h->deg = c.take<int32_t>(n);
  h->comp = c.take<int32_t>(n);
  h->anchors = c.take<int32_t>(nc);
  h->dec_anchors = c.take<int32_t>(nc);
  h->is_anchor = c.take<uint8_t>(n);
  h->inv_d = c.take<double>(n);
  h->inv_diag = c.take<double>(n);
  h->inv_d32 = c.take<float>(n);
  h->inv_diag32 = c.take<float>(n);
  h->Q0 = c.take<double>(3 * F * k);
  h->Q = c.take<double>(3 * F * k);
  h->Zb = c.take<double>(3 * F * k);
  h->U = c.take<double>(3 * F * k);
  h->V = c.take<double>(3 * k * k);
  h->H = c.take<double>(3 * k * k);
  h->G = c.take<double>(3 * k * k);
  h->Rf = c.take<double>(3 * k * k);
  h->qr_save = c.take<double>(3 * F * k);
  h->qr_bad = c.take<uint32_t>(4);
  h->theta = c.take<double>(3 * k);
  h->Wk = c.take<double>(3 * n * k);
  h->partials = c.take<double>(h->partial_elems);
  h->chg_work = c.take<double>(3 * k * k + 3 * F * k);
  h->chg = c.take<double>(3);
  h->Cf = c.take<double>(3 * k * n);
  h->qparams = c.take<double>(3 * (4 * k + 2));
  h->X = c.take<double>(n * W);
  h->D = c.take<double>(n * W);
  h->B = c.take<double>(n * W);
  h->R = c.take<double>(n * W);
  h->P = c.take<double>(n * W);
  h->Tv = c.take<double>(n * W);
  h->Qv = c.take<double>(n * W);
  h->Udeq = c.take<double>(3 * F * k);
  h->Cdeq = c.take<double>(3 * k * n);
  h->Ahat = c.take<double>(3 * nc * F);
  h->AU = c.take<double>(3 * nc * k);
  h->Eanc = c.take<double>(3 * nc * F);
  h->Ublk = c.take<double>(3 * F * k);
  h->Uhat = c.take<double>(3 * F * k);
  const size_t Fd = F <= kDirectMaxFrames ? F : 1;
  h->Rdir = c.take<double>(3 * Fd * Fd);
  h->Vdir = c.take<double>(3 * Fd * Fd);
  h->thetaF = c.take<double>(3 * Fd);
  h->cg.rz = c.take<double>(W);
  h->cg.rr = c.take<double>(W);
  h->cg.bb = c.take<double>(W);
  h->cg.pap = c.take<double>(W);
  h->cg.alpha = c.take<double>(W);
  h->cg.beta = c.take<double>(W);
  h->cg.done = c.take<int32_t>(W);
  h->cg.iters = c.take<int32_t>(W);
  h->cg.partials = c.take<double>(std::max(cg_partials_elems(h->n, h->W),
                                          cg_partials_elems(h->n, (3 * h->k + h->n_c + 3) / 4 * 4)));
  h->cg.active = c.take<int32_t>(1);
  h->cg.all_done = c.take<int32_t>(1);
  h->d_status = c.take<uint32_t>(4);
  h->d_match = c.take<int32_t>(1);
  h->ref_bb = c.take<double>(W);
  h->ref_rr = c.take<double>(W);
  h->ref_prev = c.take<double>(W);
  h->ref_t2 = c.take<double>(W);
  h->ref_frozen = c.take<int32_t>(W);
  h->ref_iters = c.take<int32_t>(W);
  size_t off = mixed_carve(h, (char*)base, c.off);
  return off + 1024;
}

int gemm_splits(long long K, long long tiles) {
  // enough split-K CTAs to cover the SMs several times, at least 64 k per split
  long long want = std::max<long long>(1, (152 * 8) / std::max<long long>(1, tiles));
  long long maxs = std::max<long long>(1, K / 64);
  return (int)std::min(want, maxs);
}

mesh_codec_status_t cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MC_OK;
  if (e == cudaErrorMemoryAllocation) return MC_E_OOM;
  return MC_E_CUDA;
}

#define MC_TRY(expr)                                  \
  do {                                                \
    cudaError_t _e = (expr);                          \
    if (_e != cudaSuccess) return cuda_status(_e);    \
  } while (0)

mesh_codec_status_t status_from_bits(uint32_t bits) {
  if (bits & ST_BAD_INDEX) return MC_E_BAD_MESH;
  if (bits & ST_DEGENERATE) return MC_E_BAD_MESH;
  if (bits & ST_ISOLATED) return MC_E_ISOLATED_VERTEX;
  if (bits & ST_BAD_ANCHORS) return MC_E_BAD_ANCHORS;
  if (bits & ST_NO_ANCHOR) return MC_E_NO_ANCHOR_IN_COMPONENT;
  if (bits & ST_BITSTREAM) return MC_E_BITSTREAM_CORRUPT;
  if (bits & ST_TC_TIMEOUT) return MC_E_TIMEOUT;
  if (bits & ST_CHOL_BREAKDOWN) return MC_E_NUMERICAL;
  if (bits & ST_NOT_CONVERGED) return MC_E_NOT_CONVERGED;
  return MC_OK;
}

mesh_codec_status_t read_status(mesh_codec* h, cudaStream_t s) {
  MC_TRY(cudaMemcpyAsync(h->h_status, h->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  MC_TRY(cudaStreamSynchronize(s));
  MC_TRY(cudaGetLastError());
  return status_from_bits(*h->h_status);
}

// positions in the caller's layout -> the vertex-major [n][3F] matrix: a
// transpose for [F][n][3] (MC_LAYOUT_FRAMES), a copy for [n][3][F]
// (MC_LAYOUT_VERTEX_MAJOR), which is the internal layout already
void ingest(const mesh_codec* h, const double* pos, double* X, cudaStream_t s, Launches& L) {
  if (h->p.layout == MC_LAYOUT_VERTEX_MAJOR)
    cudaMemcpyAsync(X, pos, sizeof(double) * 3ull * h->n * h->F, cudaMemcpyDeviceToDevice, s);
  else
    frames_to_vertex_major(pos, X, h->F, h->n, s, L);
}

// the vertex-major [n][3F] matrix -> positions in the caller's layout
void emit(const mesh_codec* h, const double* X, double* pos, cudaStream_t s, Launches& L) {
  if (h->p.layout == MC_LAYOUT_VERTEX_MAJOR)
    cudaMemcpyAsync(pos, X, sizeof(double) * 3ull * h->n * h->F, cudaMemcpyDeviceToDevice, s);
  else
    vertex_major_to_frames(X, pos, h->F, h->n, s, L);
}

bool valid_params(const mesh_codec_params_t* p) {
  if (!p) return false;
  if (p->n_vertices < 1 || p->n_triangles < 1 || p->n_frames < 1) return false;
  if (p->rank < 1 || p->rank > p->n_frames || p->rank > MESH_CODEC_MAX_RANK) return false;
  if (p->coeff_bits < 0 || p->coeff_bits > MESH_CODEC_MAX_BITS) return false;
  if (p->dict_bits < 0 || p->dict_bits > MESH_CODEC_MAX_BITS) return false;
  if (p->anchor_bits < 0 || p->anchor_bits > MESH_CODEC_MAX_BITS) return false;
  if (p->n_anchors < 0 || p->n_anchors > p->n_vertices) return false;
  if (p->laplacian_kind != 0 && p->laplacian_kind != 1) return false;
  if (p->precision < MC_PRECISION_FP64 || p->precision > MC_PRECISION_BF16) return false;
  if (p->oi_refine_sweeps < 0) return false;
  if (p->oi_sweeps < 0 || p->cg_max_iters < 1) return false;
  if (!(p->oi_tol >= 0.0) || !(p->cg_rtol >= 0.0)) return false;
  if (p->solve_mode < MC_SOLVE_FRAMES || p->solve_mode > MC_SOLVE_AUTO) return false;
  // 3F columns x n rows must be indexable, and the per-coordinate product fit
  if ((long long)p->n_frames * 3 > (1LL << 30)) return false;
  if ((long long)p->n_vertices * 3 * p->n_frames > (1LL << 40)) return false;
  if (p->autotune != 0 && p->autotune != 1) return false;
  if (p->block_delta != 0 && p->block_delta != 1) return false;
  if (p->block_delta_bits < 0 || p->block_delta_bits > MESH_CODEC_MAX_BITS) return false;
  if (p->refine < 0 || p->refine > 12) return false;
  if (p->layout != MC_LAYOUT_FRAMES && p->layout != MC_LAYOUT_VERTEX_MAJOR) return false;
  if (p->block_cg != 0 && p->block_cg != 1) return false;
  if (p->block_cg && p->refine == 0) return false;
  return true;
}

}  // namespace

extern "C" {

const char* mesh_codec_status_string(mesh_codec_status_t s) {
  switch (s) {
    case MC_OK: return "ok";
    case MC_E_INVALID_ARG: return "invalid argument";
    case MC_E_BAD_MESH: return "bad mesh (index out of range or repeated vertex)";
    case MC_E_ISOLATED_VERTEX: return "isolated vertex";
    case MC_E_OOM: return "out of memory";
    case MC_E_CUDA: return "CUDA error";
    case MC_E_NOT_CONVERGED: return "decoder solve did not converge";
    case MC_E_BITSTREAM_CORRUPT: return "corrupt bitstream";
    case MC_E_BUFFER_TOO_SMALL: return "output buffer too small";
    case MC_E_NUMERICAL: return "no orthonormal basis (non-finite data)";
    case MC_E_BAD_ANCHORS: return "bad anchor indices";
    case MC_E_NO_ANCHOR_IN_COMPONENT: return "a connected component of the mesh holds no anchor";
    case MC_E_TIMEOUT: return "a bounded device wait ran out";
  }
  return "unknown status";
}

void mesh_codec_default_params(mesh_codec_params_t* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->coeff_bits = 12;
  p->dict_bits = 16;
  p->anchor_bits = 16;
  p->laplacian_kind = 0;
  p->precision = MC_PRECISION_FP64;
  p->oi_sweeps = 30;
  p->cg_max_iters = 50000;
  p->oi_tol = 0.0;
  p->cg_rtol = 1e-14;
  p->seed = 0;
  p->solve_mode = MC_SOLVE_FRAMES;
}

void mesh_codec_destroy(mesh_codec_t* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  if (h->ws) cudaFree(h->ws);
  if (h->Gcache) cudaFree(h->Gcache);
  mc::bcg_release(h);
  if (h->Gcache_anchors) cudaFree(h->Gcache_anchors);
  if (h->Glp) cudaFree(h->Glp);
  if (h->Ahlp) cudaFree(h->Ahlp);
  if (h->stage_pos) cudaFree(h->stage_pos);
  if (h->stage_bits) cudaFree(h->stage_bits);
  if (h->h_status) cudaFreeHost(h->h_status);
  if (h->h_active) cudaFreeHost(h->h_active);
  if (h->h_header) cudaFreeHost(h->h_header);
  if (h->h_chg) cudaFreeHost(h->h_chg);
  for (cudaEvent_t e : h->prof_events) cudaEventDestroy(e);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_done) cudaEventDestroy(h->ev_done);
  if (h->ev_chunk) cudaEventDestroy(h->ev_chunk);
  if (h->own) cudaStreamDestroy(h->own);
  for (cudaGraphExec_t g : h->graph_exec)
    if (g) cudaGraphExecDestroy(g);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
}

static mesh_codec_status_t create_impl(mesh_codec* h, const int32_t* tris_in, int tris_dev,
                                       const int32_t* anchors_in, int anchors_dev,
                                       cudaStream_t s) {
  Launches L{&h->launches_create};
  const int n = h->n, T = h->T;
  h->lay = make_layout(n, h->F, h->k, h->n_c, h->p.coeff_bits, h->p.dict_bits,
                       h->p.anchor_bits, h->kind);
  h->geom = cg_geometry(n, h->W);
  // split-K partial buffer: the largest of the encoder's reductions
  {
    size_t F = h->F, k = h->k;
    int sz = gemm_splits(n, ((F + 63) / 64) * ((k + 31) / 32));
    int sh = gemm_splits(n, ((k + 63) / 64) * ((k + 31) / 32));
    int sg = gemm_splits(F, ((k + 63) / 64) * ((k + 31) / 32));
    size_t a = (size_t)sz * 3 * F * k, b = (size_t)sh * 3 * k * k, c = (size_t)sg * 3 * k * k;
    h->partial_elems = std::max(a, std::max(b, c));
    if (h->F <= kDirectMaxFrames) {   // R[1] = A A^T of the blocks variant
      const int sd = gemm_splits(n, ((F + 63) / 64) * ((F + 31) / 32));
      h->partial_elems = std::max(h->partial_elems, (size_t)sd * 3 * F * F);
    }
  }
  h->lay_delta = make_layout(n, h->F, h->k, h->n_c, h->p.coeff_bits, h->p.block_delta_bits,
                             h->p.anchor_bits, h->kind);
  mixed_dims(h);
  h->ws_bytes = carve(h, nullptr);
  MC_TRY(cudaMalloc(&h->ws, h->ws_bytes));
  carve(h, h->ws);
  if (!mixed_init(h, s)) return MC_E_CUDA;
  MC_TRY(cudaMallocHost(&h->h_status, sizeof(uint32_t) * 4));
  MC_TRY(cudaMallocHost(&h->h_active, sizeof(int32_t) * 4));
  MC_TRY(cudaMallocHost(&h->h_header, 64));
  MC_TRY(cudaMallocHost(&h->h_chg, sizeof(double) * 4));
  MC_TRY(cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking));
  MC_TRY(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  MC_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  MC_TRY(cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming));
  MC_TRY(cudaEventCreateWithFlags(&h->ev_chunk, cudaEventDisableTiming));
  MC_TRY(cudaMemsetAsync(h->d_status, 0, sizeof(uint32_t) * 4, s));

  // temporaries for the CSR build
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  {
    Carver c(nullptr);
    c.take<int32_t>(n);
    c.take<int32_t>(n + 1);
    c.take<int32_t>(n);
    c.take<int32_t>(6ull * T);
    c.take<int32_t>(scan_tmp_elems(n));
    c.take<int32_t>(3ull * T);
    c.take<int32_t>(std::max(h->n_c, 1));
    c.take<int32_t>(n);
    tmp_bytes = c.off + 256;
  }
  MC_TRY(cudaMalloc(&tmp, tmp_bytes));
  Carver c(tmp);
  CsrBuildTmp t{};
  t.raw_deg = c.take<int32_t>(n);
  t.raw_off = c.take<int32_t>(n + 1);
  t.cursor = c.take<int32_t>(n);
  t.raw_col = c.take<int32_t>(6ull * T);
  t.scan_tmp = c.take<int32_t>(scan_tmp_elems(n));
  int32_t* tris_dev_buf = c.take<int32_t>(3ull * T);
  int32_t* anchors_tmp = c.take<int32_t>(std::max(h->n_c, 1));
  int32_t* cc_parent = c.take<int32_t>(n);
  const int32_t* tris = tris_in;
  if (!tris_dev) {
    cudaError_t e = cudaMemcpyAsync(tris_dev_buf, tris_in, sizeof(int32_t) * 3ull * T,
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { cudaFree(tmp); return cuda_status(e); }
    tris = tris_dev_buf;
  }
  build_csr(tris, T, n, t, h->row_ptr, nullptr, h->deg, h->d_status, s, L);
  compact_csr(t, h->row_ptr, h->col_idx, n, s, L);
  component_labels(h->row_ptr, h->col_idx, n, cc_parent, h->comp, s, L);
  // anchors
  if (h->n_c > 0) {
    if (anchors_in) {
      const int32_t* a = anchors_in;
      if (!anchors_dev) {
        cudaError_t e = cudaMemcpyAsync(anchors_tmp, anchors_in, sizeof(int32_t) * h->n_c,
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { cudaFree(tmp); return cuda_status(e); }
        a = anchors_tmp;
      }
      cudaMemcpyAsync(h->anchors, a, sizeof(int32_t) * h->n_c, cudaMemcpyDeviceToDevice, s);
      check_anchors(h->anchors, h->n_c, n, h->d_status, s, L);
    } else {
      select_anchors(n, h->n_c, h->p.seed, h->anchors, s, L);
    }
    // Eq. 12 needs an anchor in every connected component (is_anchor: scratch here)
    anchor_coverage(h->comp, n, h->anchors, h->n_c, h->is_anchor, h->d_status, s, L);
  }
  cudaMemsetAsync(h->is_anchor, 0, n, s);
  mark_anchors(h->anchors, h->n_c, h->is_anchor, s, L);
  vertex_scalars_marked(h->row_ptr, h->col_idx, h->deg, h->is_anchor, n, h->kind, h->inv_d,
                        h->inv_diag, s, L);
  // starting basis Q0: splitmix64 uniforms made orthonormal by CholeskyQR3
  gen_start_basis(h->Q0, h->F, h->k, h->p.seed, s, L);
  int sg = gemm_splits(h->F, ((h->k + 63) / 64) * ((h->k + 31) / 32));
  cholqr3(h->Q0, h->F, h->k, qr_work(h, sg), nullptr, h->d_status, s, L);
  mesh_codec_status_t st = read_status(h, s);
  int32_t nnz = 0;
  if (st == MC_OK) {
    cudaMemcpy(&nnz, h->row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost);
    h->nnz = nnz;
    std::vector<int32_t> dg(n);
    cudaMemcpy(dg.data(), h->deg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    h->max_degree = 0;
    for (int i = 0; i < n; ++i) h->max_degree = std::max(h->max_degree, (int)dg[i]);
  }
  cudaFree(tmp);
  if (st == MC_OK) MC_TRY(cudaGetLastError());
  return st;
}

mesh_codec_status_t mesh_codec_create(const mesh_codec_params_t* params, const int32_t* triangles,
                                      int triangles_on_device, const int32_t* anchors,
                                      int anchors_on_device, void* stream, mesh_codec_t** out) {
  if (!out) return MC_E_INVALID_ARG;
  *out = nullptr;
  if (!valid_params(params) || !triangles) return MC_E_INVALID_ARG;
  mesh_codec* h = new (std::nothrow) mesh_codec();
  if (!h) return MC_E_OOM;
  h->p = *params;
  h->n = params->n_vertices;
  h->T = params->n_triangles;
  h->F = params->n_frames;
  h->k = params->rank;
  h->W = 3 * h->F;
  h->n_c = params->n_anchors;
  h->kind = params->laplacian_kind;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  mesh_codec_status_t st = create_impl(h, triangles, triangles_on_device, anchors,
                                       anchors_on_device, s);
  if (st != MC_OK) {
    mesh_codec_destroy(h);
    return st;
  }
  *out = h;
  return MC_OK;
}

mesh_codec_status_t mesh_codec_encoded_size(const mesh_codec_t* h, size_t* bytes) {
  if (!h || !bytes) return MC_E_INVALID_ARG;
  *bytes = (size_t)h->lay.total;
  return MC_OK;
}

// Options of one encode: the blocks variant supplies the start basis or the
// direct eigendecomposition (Algorithm 1), a dictionary reference for the
// difference coding of consecutive dictionaries, and that stream's layout.
struct EncodeOpts {
  const double* start = nullptr;       // start basis [3][F][k]; null: the handle's Q0
  bool direct = false;                 // U = top-k eigenvectors of A A^T (F <= 64)
  const double* dict_ref = nullptr;    // dictionary section codes U - dict_ref
  const EncodeLayout* lay = nullptr;   // null: the handle's layout
};

__global__ void k_take_cols(const double* __restrict__ V, int rows, int ld, int cols,
                            double* __restrict__ U) {
  // U[c][r][j] = V[c][r][j] for j < cols (V: [3][rows][ld])
  const long long total = 3LL * rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / ((long long)rows * cols), rem = e % ((long long)rows * cols);
    U[e] = V[(c * rows + rem / cols) * ld + rem % cols];
  }
}

__global__ void k_axpy_sub(const double* __restrict__ a, const double* __restrict__ b,
                           long long count, double sign, double* __restrict__ out) {
  // out = a + sign * b (sign = -1: the coded difference; +1: the reconstruction)
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = sign > 0 ? __dadd_rn(a[e], b[e]) : __dsub_rn(a[e], b[e]);
}

// B[anchors[a]][c*k + j] += AU[c][a][j]: P^T (A^_c U'_c) into the data columns
__global__ void k_scatter_anchor_proj(double* B, const double* __restrict__ AU,
                                      const int32_t* __restrict__ anchors, int n_c, int k, int Wc) {
  const long long total = 3LL * n_c * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / ((long long)n_c * k), rem = e % ((long long)n_c * k);
    const long long a = rem / k, j = rem % k;
    B[(long long)anchors[a] * Wc + c * k + j] += AU[e];
  }
}

static void scatter_anchor_proj(double* B, const double* AU, const int32_t* anchors, int n_c,
                                int k, int Wc, cudaStream_t s, Launches& L) {
  const long long total = 3LL * n_c * k;
  k_scatter_anchor_proj<<<(int)std::min<long long>((total + 255) / 256, 1024), 256, 0, s>>>(
      B, AU, anchors, n_c, k, Wc);
  L.add(1);
}

static void enqueue_encode(mesh_codec* h, const double* positions, uint8_t* out, cudaStream_t s,
                           Launches& L, bool host_check_tol, const EncodeOpts& o = EncodeOpts()) {
  const int n = h->n, F = h->F, k = h->k, W = h->W;
  const EncodeLayout& lay = o.lay ? *o.lay : h->lay;
  cudaMemsetAsync(h->d_status, 0, sizeof(uint32_t), s);
  ingest(h, positions, h->X, s, L);
  laplacian_rows(h->row_ptr, h->col_idx, h->deg, h->X, h->D, n, W, h->kind, s, L);

  // orthogonal iterations, three coordinates batched
  const Strided Xc{h->X, W, 1, F};        // A_c^T (n x F): element (i, f)
  const Strided XcT{h->X, 1, W, F};       // A_c (F x n): element (f, i)
  const int sz = gemm_splits(n, ((F + 63) / 64) * ((k + 31) / 32));
  const int sh = gemm_splits(n, ((k + 63) / 64) * ((k + 31) / 32));
  const int sg = gemm_splits(F, ((k + 63) / 64) * ((k + 31) / 32));
  for (int c = 0; c < 3; ++c) { h->oi_done[c] = 0; h->oi_last_change[c] = 0.0; }
  if (o.direct) {
    // Algorithm 1's first block: R = A_c A_c^T (F x F), its eigenvectors
    // descending (Jacobi), the first k of them, signs
    const int sd = gemm_splits(n, ((F + 63) / 64) * ((F + 31) / 32));
    dgemm(F, F, n, 3, XcT, Xc, StridedOut{h->Rdir, F, 1, (long long)F * F}, sd, h->partials, s,
          L);
    jacobi_eig(h->Rdir, h->Vdir, h->thetaF, F, s, L);
    k_take_cols<<<(3 * F * k + 255) / 256, 256, 0, s>>>(h->Vdir, F, F, k, h->U);
    k_take_cols<<<1, 256, 0, s>>>(h->thetaF, 1, F, k, h->theta);
    L.add(2);
    sign_rule(h->U, F, k, s, L);
  } else {
  cudaMemcpyAsync(h->Q, o.start ? o.start : h->Q0, sizeof(double) * 3 * F * k,
                  cudaMemcpyDeviceToDevice, s);
  // mixed precision: tensor-core sweeps first, then the FP64 refinement sweeps
  int fp64_sweeps = h->p.oi_sweeps;
  if (h->lp >= 0) {
    mixed_oi_sweeps(h, h->p.oi_sweeps, s, L);
    fp64_sweeps = h->p.oi_refine_sweeps;
  }
  for (int t = 0; t < fp64_sweeps; ++t) {
    dgemm(n, k, F, 3, Xc, Strided{h->Q, k, 1, (long long)F * k},
          StridedOut{h->Wk, k, 1, (long long)n * k}, 1, nullptr, s, L);
    dgemm(F, k, n, 3, XcT, Strided{h->Wk, k, 1, (long long)n * k},
          StridedOut{h->Zb, k, 1, (long long)F * k}, sz, h->partials, s, L);
    cholqr3(h->Zb, F, k, qr_work(h, sg), h->Q, h->d_status, s, L);
    for (int c = 0; c < 3; ++c) h->oi_done[c] = t + 1;
    bool stop = false;
    if (host_check_tol && h->p.oi_tol > 0.0) {
      oi_change(h->Q, h->Zb, F, k, h->chg_work, h->chg, s, L);
      cudaMemcpyAsync(h->h_chg, h->chg, sizeof(double) * 3, cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      stop = true;
      for (int c = 0; c < 3; ++c) {
        h->oi_last_change[c] = h->h_chg[c];
        stop = stop && (h->h_chg[c] <= h->p.oi_tol);
      }
    }
    std::swap(h->Q, h->Zb);
    if (stop) break;
  }
  // Rayleigh-Ritz: H = (A_c^T Q)^T (A_c^T Q), eigenvectors V, U = Q V, signs
  dgemm(n, k, F, 3, Xc, Strided{h->Q, k, 1, (long long)F * k},
        StridedOut{h->Wk, k, 1, (long long)n * k}, 1, nullptr, s, L);
  dgemm(k, k, n, 3, Strided{h->Wk, 1, k, (long long)n * k}, Strided{h->Wk, k, 1, (long long)n * k},
        StridedOut{h->H, k, 1, (long long)k * k}, sh, h->partials, s, L);
  jacobi_eig(h->H, h->V, h->theta, k, s, L);
  dgemm(F, k, k, 3, Strided{h->Q, k, 1, (long long)F * k}, Strided{h->V, k, 1, (long long)k * k},
        StridedOut{h->U, k, 1, (long long)F * k}, 1, nullptr, s, L);
  sign_rule(h->U, F, k, s, L);
  }
  // projection C_c = U_c^T delta_c^T (k x n); with the refined solve it stays
  // FP64, so that only the orthogonal-iteration sweeps (which the FP64
  // refinement sweep and Rayleigh-Ritz correct) use the tensor cores
  if (h->lp >= 0 && h->p.refine == 0) {
    mixed_project(h, s, L);
  } else {
    dgemm(k, n, F, 3, Strided{h->U, 1, k, (long long)F * k}, Strided{h->D, 1, W, F},
          StridedOut{h->Cf, n, 1, (long long)k * n}, 1, nullptr, s, L);
  }
  // the coded dictionary: U, or its difference from the reference (into Zb,
  // free after the sweeps)
  const double* Ucode = h->U;
  if (o.dict_ref) {
    const long long cnt = 3LL * F * k;
    k_axpy_sub<<<(int)std::min<long long>((cnt + 255) / 256, 1024), 256, 0, s>>>(
        h->U, o.dict_ref, cnt, -1.0, h->Zb);
    L.add(1);
    Ucode = h->Zb;
  }
  // quantizer ranges: dictionary columns, coefficient rows, anchors
  const long long P = 4LL * k + 2;
  minmax_rows_out(Ucode, k, F, 1, k, 3, (long long)F * k, h->qparams, h->qparams + k, P, s, L);
  minmax_rows_out(h->Cf, k, n, n, 1, 3, (long long)k * n, h->qparams + 2 * k, h->qparams + 3 * k,
                  P, s, L);
  anchor_minmax_out(h->X, h->anchors, h->n_c, F, h->qparams + 4 * k, h->qparams + 4 * k + 1, P,
                    s, L);
  write_header(out, lay, h->anchors, h->qparams, s, L);
  quant_pack_sections(out, lay, Ucode, h->Cf, h->X, h->anchors, h->qparams, s, L);
}

mesh_codec_status_t mesh_codec_encode(mesh_codec_t* h, const double* positions, uint8_t* bitstream,
                                      size_t capacity, size_t* written, void* stream) {
  if (!h || !positions || !bitstream || !written) return MC_E_INVALID_ARG;
  if (((uintptr_t)bitstream & 7) || ((uintptr_t)positions & 7)) return MC_E_INVALID_ARG;
  *written = (size_t)h->lay.total;
  if (capacity < (size_t)h->lay.total) return MC_E_BUFFER_TOO_SMALL;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  h->launches_encode = 0;
  Launches L{&h->launches_encode};
  enqueue_encode(h, positions, bitstream, s, L, true);
  MC_TRY(cudaGetLastError());
  return read_status(h, s);
}

static mesh_codec_status_t check_header(mesh_codec* h, const uint8_t* hdr, size_t bytes,
                                        const EncodeLayout* lay = nullptr) {
  uint32_t w[8];
  std::memcpy(w, hdr, 32);
  unsigned long long total;
  std::memcpy(&total, hdr + 32, 8);
  const EncodeLayout& L = lay ? *lay : h->lay;
  if (w[0] != 0x31434D44u || w[1] != 1u || w[7] != 64u) return MC_E_BITSTREAM_CORRUPT;
  if ((int)w[2] != L.n || (int)w[3] != L.F || (int)w[4] != L.k || (int)w[5] != L.n_c)
    return MC_E_BITSTREAM_CORRUPT;
  if (hdr[24] != L.cb || hdr[25] != L.db || hdr[26] != L.ab || hdr[27] != L.kind)
    return MC_E_BITSTREAM_CORRUPT;
  if (total != (unsigned long long)L.total || bytes != (size_t)L.total)
    return MC_E_BITSTREAM_CORRUPT;
  return MC_OK;
}

// events for CG iteration `it` when profiling samples it, else null
static cudaEvent_t* prof_group(mesh_codec* h, int it) {
  if (h->prof_every <= 0 || it % h->prof_every != 0) return nullptr;
  const size_t G = kCgKernels + 1;
  if ((h->prof_used + 1) * G > h->prof_events.size()) {
    for (size_t i = 0; i < G; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      h->prof_events.push_back(e);
    }
  }
  return &h->prof_events[(h->prof_used++) * G];
}

// an event pair around a run of `iters` CG iterations when timing is on, else null
static cudaEvent_t* prof_run(mesh_codec* h, int iters) {
  if (h->prof_every <= 0) return nullptr;
  if ((h->run_used + 1) * 2 > h->run_events.size()) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      h->run_events.push_back(e);
    }
  }
  if (h->run_iters.size() < h->run_used + 1) h->run_iters.resize(h->run_used + 1);
  h->run_iters[h->run_used] = iters;
  return &h->run_events[(h->run_used++) * 2];
}

// after the decode's final synchronisation: fold the recorded groups into totals
static void prof_collect(mesh_codec* h) {
  for (size_t g = 0; g < h->run_used; ++g) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->run_events[2 * g], h->run_events[2 * g + 1]) ==
        cudaSuccess) {
      h->prof_ms[kCgKernels] += ms;
      h->prof_launches[kCgKernels] += h->run_iters[g];
    }
  }
  h->run_used = 0;
  const size_t G = kCgKernels + 1;
  for (size_t g = 0; g < h->prof_used; ++g) {
    for (int k = 0; k < kCgKernels; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->prof_events[g * G + k], h->prof_events[g * G + k + 1]) ==
          cudaSuccess) {
        h->prof_ms[k] += ms;
        h->prof_launches[k] += 1;
      }
    }
  }
  h->prof_used = 0;
}

// the factored decode solves 3k + n_c columns instead of 3F
static bool use_factored(const mesh_codec* h) {
  if (h->p.solve_mode == MC_SOLVE_FACTORED) return true;
  if (h->p.solve_mode == MC_SOLVE_AUTO) return 3 * h->k + h->n_c < 3 * h->F;
  return false;
}

__global__ void k_flag_not_converged(const int32_t* done, int W, uint32_t* status);

// *count += number of positions where a and b differ
__global__ void k_count_mismatch(const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                                 int count, int32_t* out) {
  int diff = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    diff += a[i] != b[i];
  if (diff) atomicAdd(out, diff);
}

// G[i][a] = X[i][col0 + a] for a < cols (X: [n][ld])
__global__ void k_copy_cols(const double* __restrict__ X, int ld, int col0, int n, int cols,
                            double* __restrict__ G) {
  const long long total = (long long)n * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    G[e] = X[(e / cols) * ld + col0 + e % cols];
}

// the kept anchor response becomes usable once its decode converged
static void settle_anchor_cache(mesh_codec* h, mesh_codec_status_t st) {
  if (h->Gcache_pending) h->Gcache_valid = st == MC_OK;
  h->Gcache_pending = false;
}

// Decoder, in three phases so that several handles can advance their CG
// solves in lockstep on their own streams (mesh_codec_decode_batch).
// Phase 1: unpack, back-projection, right-hand sides, CG start.
static void decode_prepare(mesh_codec* h, const uint8_t* in, cudaStream_t s, Launches& L,
                           const double* x0 = nullptr, const double* dict_ref = nullptr,
                           const EncodeLayout* lay = nullptr) {
  const int n = h->n, F = h->F, k = h->k, W = h->W;
  DecodeState& d = h->dec;
  cudaMemsetAsync(h->d_status, 0, sizeof(uint32_t), s);
  unpack_sections(in, lay ? *lay : h->lay, h->Udeq, h->Cdeq, h->Ahat, h->dec_anchors, nullptr,
                  h->d_status, s, L);
  if (dict_ref) {   // the dictionary section holds differences from dict_ref
    const long long cnt = 3LL * F * k;
    k_axpy_sub<<<(int)std::min<long long>((cnt + 255) / 256, 1024), 256, 0, s>>>(
        h->Udeq, dict_ref, cnt, 1.0, h->Udeq);
    L.add(1);
  }
  // the decoder's anchor set comes from the stream
  cudaMemsetAsync(h->is_anchor, 0, n, s);
  mark_anchors(h->dec_anchors, h->n_c, h->is_anchor, s, L);
  vertex_scalars_marked(h->row_ptr, h->col_idx, h->deg, h->is_anchor, n, h->kind, h->inv_d,
                        h->inv_diag, s, L);
  d.factored = use_factored(h);
  // the kept anchor response applies when this stream's anchors are its
  // anchors; in the automatic mode, anchors that repeat the previous decode's
  // make the factored solve worth its extra n_c columns once (its G then
  // serves every later decode), unless a first iterate asks for the frames solve
  const bool automatic = h->p.solve_mode == MC_SOLVE_AUTO && x0 == nullptr;
  d.cached = false;
  bool repeat = false;
  if (h->n_c > 0 && ((d.factored && h->Gcache_valid) || (automatic && h->anchors_kept))) {
    cudaMemsetAsync(h->d_match, 0, sizeof(int32_t), s);
    k_count_mismatch<<<(h->n_c + 255) / 256, 256, 0, s>>>(h->dec_anchors, h->Gcache_anchors,
                                                          h->n_c, h->d_match);
    L.add(1);
    cudaMemcpyAsync(h->h_active + 1, h->d_match, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    repeat = h->h_active[1] == 0;
  }
  if (repeat && h->Gcache_valid) {
    d.factored = true;
    d.cached = true;
  } else if (repeat && automatic) {
    d.factored = true;
  }
  d.store = d.factored && !d.cached;
  if (automatic && !d.factored && h->n_c > 0) {
    // keep this decode's anchors (a G kept for other anchors no longer applies)
    if (!h->Gcache_anchors &&
        cudaMalloc(&h->Gcache_anchors, sizeof(int32_t) * h->n_c) != cudaSuccess) {
      cudaGetLastError();
      h->Gcache_anchors = nullptr;
    }
    if (h->Gcache_anchors) {
      cudaMemcpyAsync(h->Gcache_anchors, h->dec_anchors, sizeof(int32_t) * h->n_c,
                      cudaMemcpyDeviceToDevice, s);
      h->Gcache_valid = false;
      h->anchors_kept = true;
    }
  }
  // CG columns: 3F frames (Eq. 11-12 as written), or 3k + n_c factored columns,
  // or the 3k data columns with the kept anchor response (the FP32 factored
  // solve and the block CG pad the column count to a multiple of 4 with zero
  // right-hand sides, which converge at once, for the float4 kernels)
  d.Wc = d.factored ? (d.cached ? 3 * k : 3 * k + h->n_c) : W;
  if (d.factored && (h->lp >= 0 || h->p.block_cg)) d.Wc = (d.Wc + 3) / 4 * 4;
  if (!d.factored) {
    // delta~_c = (U_c' C_c')^T : (n x k)(k x F) into D[:, cF : cF + F]
    if (h->lp >= 0 && h->p.refine == 0) {
      mixed_backproject(h, s, L);
    } else {
      dgemm(n, F, k, 3, Strided{h->Cdeq, 1, n, (long long)k * n},
            Strided{h->Udeq, 1, k, (long long)F * k}, StridedOut{h->D, W, 1, F}, 1, nullptr, s,
            L);
    }
    // B = L^T delta~ + P^T a^
    laplacian_t_rows(h->row_ptr, h->col_idx, h->deg, h->inv_d, h->D, h->B, n, W, h->kind, s, L);
    for (int c = 0; c < 3; ++c)
      scatter_anchor_rhs(h->B, h->Ahat + (long long)c * std::max(h->n_c, 1) * F, h->dec_anchors,
                         h->n_c, F, W, c * F, s, L);
  } else {
    // E = [C_x'^T | C_y'^T | C_z'^T | 0] (n x Wc); B = L^T E, then column 3k + a of B
    // gets e_{anchor a}:  M Y = L^T C'^T and M G = P^T
    factored_rhs(h->Cdeq, k, n, d.Wc, h->D, s, L);
    laplacian_t_rows(h->row_ptr, h->col_idx, h->deg, h->inv_d, h->D, h->B, n, d.Wc, h->kind, s,
                     L);
    if (!d.cached) unit_anchor_columns(h->B, h->dec_anchors, h->n_c, d.Wc, 3 * k, s, L);
    if (h->lp >= 0 && h->n_c > 0) {
      // mixed modes: A^_c = (A^_c U'_c) U'_c^T + E_c, so the data columns also
      // carry P^T A^_c U'_c and G multiplies only the small residual E_c (the
      // part of the anchors' trajectories outside the dictionary), which the
      // tensor cores then form with an error relative to E_c, not to A^_c
      const long long nc = h->n_c;
      dgemm((int)nc, k, F, 3, Strided{h->Ahat, F, 1, nc * F}, Strided{h->Udeq, k, 1, (long long)F * k},
            StridedOut{h->AU, k, 1, nc * k}, 1, nullptr, s, L);
      scatter_anchor_proj(h->B, h->AU, h->dec_anchors, h->n_c, k, d.Wc, s, L);
    }
  }
  // CG: FP64 vectors, or FP32 vectors with FP64-accurate dot products in the mixed modes
  // and for the corrections of the refined solve
  d.refine = h->p.refine > 0;
  d.single = (h->lp >= 0 || d.refine) ? 1 : 0;
  d.inv_d = h->inv_d;
  d.inv_diag = h->inv_diag;
  if (d.single) {   // FP32 copies: no FP64 conversions in the FP32 kernels
    narrow(h->inv_d, n, h->inv_d32, s, L);
    narrow(h->inv_diag, n, h->inv_diag32, s, L);
    d.inv_d = h->inv_d32;
    d.inv_diag = h->inv_diag32;
  }
  d.geom = cg_geometry(n, d.Wc);
  if (h->p.autotune) {
    if (h->tuned_W != d.Wc || h->tuned_single != d.single) {
      h->tuned = cg_autotune(n, d.Wc, h->row_ptr, h->col_idx, h->deg, d.inv_d, h->is_anchor,
                             h->kind, h->P, h->Tv, h->Qv, h->cg, d.single, s, L);
      h->tuned_W = d.Wc;
      h->tuned_single = d.single;
    }
    d.geom = h->tuned;
  }
  {
    // the FP32 operator kernels stage each row block's CSR slice in shared
    // memory when it fits a modest budget (12 KB)
    const long long cap = (long long)d.geom.rows_per_block * std::max(h->max_degree, 1);
    d.geom.csr_cap = (cap + d.geom.rows_per_block + 1) * 4 <= 12 * 1024 ? (int)cap : 0;
  }
  if (d.refine) {
    // the refined solve keeps its iterate in FP64 (X), from X0 or zero
    if (x0 && !d.factored)
      ingest(h, x0, h->X, s, L);
    else
      cudaMemsetAsync(h->X, 0, sizeof(double) * (size_t)n * d.Wc, s);
  } else if (x0 && !d.factored) {
    // warm start: the caller's X0 [F][n][3] as the CG's first iterate
    ingest(h, x0, h->D, s, L);
    if (d.single)
      narrow(h->D, (long long)n * W, (float*)h->X, s, L);
    else
      cudaMemcpyAsync(h->X, h->D, sizeof(double) * n * W, cudaMemcpyDeviceToDevice, s);
    cg_init_warm(d.geom, h->row_ptr, h->col_idx, h->deg, d.inv_d, h->is_anchor, h->kind, h->B,
                 h->X, h->R, h->P, h->Tv, h->Qv, d.inv_diag, h->cg, d.single, s, L);
  } else {
    cg_init(d.geom, h->B, h->X, h->R, h->P, d.inv_diag, h->cg, d.single, s, L);
  }
  h->cg_columns = d.Wc;
  d.it = 0;
}

// Phase 2: up to `m` CG iterations, then an asynchronous copy of the number
// of still active columns to pinned host memory.  Returns false when the
// iteration cap has been reached.
// A full chunk of CG iterations is replayed from a CUDA graph captured once
// per (column count, precision, tile shape): one launch instead of six per
// iteration.  With kernel timing on (mesh_codec_set_profiling) the chunk's
// first iteration runs as direct launches between CUDA events and the other
// kCgChunk - 1 come from a second graph, so timing samples one iteration in
// kCgChunk without giving up the graph replay.
static constexpr int kCgChunk = 32;

static bool chunk_graph(mesh_codec* h, int slot, int len) {
  const DecodeState& d = h->dec;
  if (h->graph_exec[slot] && h->graph_W[slot] == d.Wc && h->graph_single[slot] == d.single &&
      h->graph_rpb[slot] == d.geom.rows_per_block)
    return true;
  if (h->graph_exec[slot]) {
    cudaGraphExecDestroy(h->graph_exec[slot]);
    h->graph_exec[slot] = nullptr;
  }
  if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  Launches none{nullptr};
  for (int j = 0; j < len; ++j)
    cg_iteration(d.geom, h->row_ptr, h->col_idx, h->deg, d.inv_d, h->is_anchor, d.inv_diag,
                 h->kind, h->X, h->R, h->P, h->Tv, h->Qv, h->p.cg_rtol, h->p.cg_max_iters, h->cg,
                 d.single, h->cap, none, nullptr);
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(h->cap, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    return false;
  }
  cudaError_t e = cudaGraphInstantiate(&h->graph_exec[slot], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph_exec[slot] = nullptr;
    cudaGetLastError();
    return false;
  }
  h->graph_W[slot] = d.Wc;
  h->graph_single[slot] = d.single;
  h->graph_rpb[slot] = d.geom.rows_per_block;
  return true;
}

static bool decode_cg_chunk(mesh_codec* h, int m, cudaStream_t s, Launches& L) {
  DecodeState& d = h->dec;
  m = std::min(m, h->p.cg_max_iters - d.it);
  if (m <= 0) return false;
  if (m == kCgChunk && h->prof_every == 0 && chunk_graph(h, 0, kCgChunk)) {
    cudaGraphLaunch(h->graph_exec[0], s);
    L.add(6 * kCgChunk);
  } else if (m == kCgChunk && h->prof_every > 0 && chunk_graph(h, 1, kCgChunk - 1)) {
    // the chunk's timed iteration comes last: its launches queue behind the
    // graph, so no idle gap after the host's convergence check enters its
    // first kernel (the chunk is chosen by its first iteration's index); the
    // graph itself is bracketed by one event pair (its iterations' time)
    cudaEvent_t* run = prof_run(h, kCgChunk - 1);
    if (run) cudaEventRecord(run[0], s);
    cudaGraphLaunch(h->graph_exec[1], s);
    if (run) cudaEventRecord(run[1], s);
    L.add(6 * (kCgChunk - 1));
    cg_iteration(d.geom, h->row_ptr, h->col_idx, h->deg, d.inv_d, h->is_anchor, d.inv_diag,
                 h->kind, h->X, h->R, h->P, h->Tv, h->Qv, h->p.cg_rtol, h->p.cg_max_iters, h->cg,
                 d.single, s, L, prof_group(h, d.it));
  } else {
    for (int j = 0; j < m; ++j)
      cg_iteration(d.geom, h->row_ptr, h->col_idx, h->deg, d.inv_d, h->is_anchor, d.inv_diag,
                   h->kind, h->X, h->R, h->P, h->Tv, h->Qv, h->p.cg_rtol, h->p.cg_max_iters,
                   h->cg, d.single, s, L, prof_group(h, d.it + j));
  }
  d.it += m;
  cudaMemcpyAsync(h->h_active, h->cg.active, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  return true;
}

// Refined solve: outer steps X += D with D the FP32 CG solution of M D = R,
// R = B - M X formed in FP64, until every column's ||R|| <= cg_rtol ||B||.
// The inner CG reduces each correction's residual by 10^-refine; the FP32
// vectors sit in buffers the solve leaves free (X holds the FP64 iterate,
// Tv and Qv the FP64 products, R / P / D the FP32 vectors).
static constexpr int kRefineMaxOuter = 30;

static mesh_codec_status_t decode_refine(mesh_codec* h, cudaStream_t s, Launches& L) {
  DecodeState& d = h->dec;
  const int n = h->n, W = d.Wc;
  const long long nw = (long long)n * W;
  const CgGeom g64 = cg_geometry(n, W);   // the FP64 residual kernels (32 columns per CTA)
  double* X64 = h->X;
  double* T64 = h->Tv;
  double* Rres = h->Qv;
  float* X32 = (float*)h->R;
  float* R32 = X32 + nw;
  float* P32 = (float*)h->P;
  float* T32 = P32 + nw;
  float* Q32 = (float*)h->D;
  const double inner_rtol = std::pow(10.0, -(double)h->p.refine);
  // the smallest residual binary64 resolves for an iterate X: a multiple of
  // eps sqrt(n) ||M||_inf ||X|| (||M||_inf <= ||L||_inf ||L||_1 + 1)
  const double dm = (double)std::max(h->max_degree, 1);
  const double normM = h->kind == 0 ? 2.0 * (1.0 + dm) + 1.0 : 4.0 * dm * dm + 1.0;
  const double floor = 100.0 * 0x1.0p-53 * std::sqrt((double)n) * normM;
  cudaMemsetAsync(h->ref_frozen, 0, sizeof(int32_t) * W, s);
  cudaMemsetAsync(h->ref_iters, 0, sizeof(int32_t) * W, s);
  refine_reset(h->ref_prev, W, s, L);
  refine_col_norms(g64, h->B, h->cg.partials, h->ref_bb, s, L);
  for (int outer = 0;; ++outer) {
    refine_residual(g64, h->row_ptr, h->col_idx, h->deg, h->inv_d, h->is_anchor, h->kind, X64,
                    h->B, T64, Rres, h->ref_frozen, h->cg.partials, h->ref_bb, h->p.cg_rtol,
                    floor, h->ref_prev, h->ref_rr, h->cg.active, s, L);
    MC_TRY(cudaMemcpyAsync(h->h_active, h->cg.active, sizeof(int32_t), cudaMemcpyDeviceToHost,
                           s));
    MC_TRY(cudaStreamSynchronize(s));
    if (*h->h_active == 0 || outer == kRefineMaxOuter) break;
    // FP32 correction (frozen columns have R = 0 and converge at once)
    // each correction gets at most an eighth of the iteration cap (at least
    // 1000): a column whose FP32 correction cannot reach the inner tolerance
    // moves on to the next outer step instead of spinning
    const int inner_max = std::max(1000, h->p.cg_max_iters / 8);
    if (h->p.block_cg && W % 4 == 0) {
      refine_targets(h->ref_rr, h->ref_bb, h->ref_frozen, W, h->p.cg_rtol, inner_rtol,
                     h->ref_t2, nullptr, s, L);
      const int ran = bcg_solve(h, d.geom, (const float*)d.inv_d, (const float*)d.inv_diag, Rres,
                                X32, R32, P32, T32, Q32, h->cg.iters, inner_rtol, h->ref_t2,
                                inner_max, s, L);
      if (ran < 0) return MC_E_CUDA;
      d.it += ran;
      refine_update(X32, nw, X64, h->cg.iters, W, h->ref_iters, s, L);
      continue;
    }
    cg_init(d.geom, Rres, X32, R32, P32, d.inv_diag, h->cg, 1, s, L);
    refine_targets(h->ref_rr, h->ref_bb, h->ref_frozen, W, h->p.cg_rtol, inner_rtol, h->ref_t2,
                   h->cg.bb, s, L);
    for (int it = 0; it < inner_max; it += kCgChunk) {
      const int m = std::min(kCgChunk, inner_max - it);
      // timing: the first m - 1 iterations as one run, the last one per kernel
      // (sampled when the run's first iteration index is a multiple of `every`)
      cudaEvent_t* run = m > 1 ? prof_run(h, m - 1) : nullptr;
      if (run) cudaEventRecord(run[0], s);
      const int it0 = d.it;
      for (int j = 0; j < m; ++j, ++d.it) {
        const bool last = j == m - 1;
        cg_iteration(d.geom, h->row_ptr, h->col_idx, h->deg, d.inv_d, h->is_anchor, d.inv_diag,
                     h->kind, X32, R32, P32, T32, Q32, inner_rtol, inner_max, h->cg, 1, s, L,
                     last ? prof_group(h, it0) : nullptr);
        if (run && j == m - 2) cudaEventRecord(run[1], s);
      }
      MC_TRY(cudaMemcpyAsync(h->h_active, h->cg.active, sizeof(int32_t),
                             cudaMemcpyDeviceToHost, s));
      MC_TRY(cudaStreamSynchronize(s));
      if (*h->h_active == 0) break;
    }
    refine_update(X32, nw, X64, h->cg.iters, W, h->ref_iters, s, L);
  }
  // per-column results in the CG state: converged = frozen, iterations, ||R||, ||B||
  MC_TRY(cudaMemcpyAsync(h->cg.done, h->ref_frozen, sizeof(int32_t) * W,
                         cudaMemcpyDeviceToDevice, s));
  MC_TRY(cudaMemcpyAsync(h->cg.iters, h->ref_iters, sizeof(int32_t) * W,
                         cudaMemcpyDeviceToDevice, s));
  MC_TRY(cudaMemcpyAsync(h->cg.rr, h->ref_rr, sizeof(double) * W, cudaMemcpyDeviceToDevice, s));
  MC_TRY(cudaMemcpyAsync(h->cg.bb, h->ref_bb, sizeof(double) * W, cudaMemcpyDeviceToDevice, s));
  return MC_OK;
}

// Phase 3: the solution in FP64, the factored combination, the output layout.
static void decode_finish(mesh_codec* h, double* out, cudaStream_t s, Launches& L) {
  const int n = h->n, F = h->F, k = h->k, W = h->W;
  const DecodeState& d = h->dec;
  const double* Xs = h->X;
  if (d.single && !d.refine) {   // the mixed modes widen their FP32 iterate into B
    widen((const float*)h->X, (long long)n * d.Wc, h->B, s, L);
    Xs = h->B;
  }
  if (!d.factored) {
    emit(h, Xs, out, s, L);
  } else {
    // X_c = Y_c U_c'^T + G A^_c into D [n][3F]: on the tensor cores in the mixed
    // modes (FP32 solve), in FP64 otherwise (and for the refined solve)
    const double* Gp = d.cached ? h->Gcache : Xs + 3 * k;
    const long long g_ld = d.cached ? h->n_c : d.Wc;
    const long long ncs = std::max(h->n_c, 1);
    // the anchors' term G A: in the mixed modes A = E_c, the residual of the
    // anchors' trajectories outside the dictionary (see decode_prepare)
    const double* Aterm = h->Ahat;
    if (h->lp >= 0 && h->n_c > 0) {
      const long long nc = h->n_c;
      dgemm((int)nc, F, k, 3, Strided{h->AU, k, 1, nc * k}, Strided{h->Udeq, 1, k, (long long)F * k},
            StridedOut{h->Eanc, F, 1, nc * F}, 1, nullptr, s, L);
      const long long cnt = 3 * nc * F;
      k_axpy_sub<<<(int)std::min<long long>((cnt + 255) / 256, 1024), 256, 0, s>>>(
          h->Ahat, h->Eanc, cnt, -1.0, h->Eanc);
      L.add(1);
      Aterm = h->Eanc;
    }
    // plain mixed modes: both products on the tensor cores; refined solve: the
    // data product in FP64, the anchors' residual product on the tensor cores
    bool data_done = false, anchor_done = false;
    if (d.single && h->lp >= 0) {
      if (!d.refine) {
        data_done = anchor_done = mixed_finish(h, Xs, d.Wc, Gp, g_ld, Aterm, true, s, L);
      } else {
        dgemm(n, F, k, 3, Strided{Xs, d.Wc, 1, k}, Strided{h->Udeq, 1, k, (long long)F * k},
              StridedOut{h->D, W, 1, F}, 1, nullptr, s, L);
        data_done = true;
        anchor_done = mixed_finish(h, Xs, d.Wc, Gp, g_ld, Aterm, false, s, L);
      }
    }
    if (!data_done)
      dgemm(n, F, k, 3, Strided{Xs, d.Wc, 1, k}, Strided{h->Udeq, 1, k, (long long)F * k},
            StridedOut{h->D, W, 1, F}, 1, nullptr, s, L);
    if (!anchor_done) {
      StridedOut acc{h->D, W, 1, F};
      acc.accumulate = 1;
      dgemm(n, F, h->n_c, 3, Strided{Gp, g_ld, 1, 0}, Strided{Aterm, F, 1, ncs * F}, acc, 1,
            nullptr, s, L);
    }
    emit(h, h->D, out, s, L);
    if (d.store) {
      // keep G and its anchors; valid once the decode reports every column converged
      if (!h->Gcache_anchors &&
          cudaMalloc(&h->Gcache_anchors, sizeof(int32_t) * h->n_c) != cudaSuccess) {
        cudaGetLastError();
        h->Gcache_anchors = nullptr;
      }
      if (!h->Gcache && h->Gcache_anchors &&
          cudaMalloc(&h->Gcache, sizeof(double) * (size_t)n * h->n_c) != cudaSuccess) {
        cudaGetLastError();
        h->Gcache = nullptr;
      }
      if (h->Gcache) {
        h->Gcache_valid = false;
        const long long cnt = (long long)n * h->n_c;
        k_copy_cols<<<(int)std::min<long long>((cnt + 255) / 256, 4096), 256, 0, s>>>(
            Xs, d.Wc, 3 * k, n, h->n_c, h->Gcache);
        cudaMemcpyAsync(h->Gcache_anchors, h->dec_anchors, sizeof(int32_t) * h->n_c,
                        cudaMemcpyDeviceToDevice, s);
        L.add(1);
        h->Gcache_pending = true;
        h->anchors_kept = true;
      }
    }
  }
  k_flag_not_converged<<<(h->cg_columns + 255) / 256, 256, 0, s>>>(h->cg.done, h->cg_columns,
                                                                     h->d_status);
  L.add(1);
}

// The stream's anchor set (its n_c indices right after the 64-byte header,
// which the caller has checked) must hold an anchor in every connected
// component of the mesh, or Eq. 12 is singular.  Enqueues the check and the
// copy of its result word to pinned memory; is_anchor serves as scratch (the
// decoder rebuilds it from the stream).
static void enqueue_anchor_check(mesh_codec* h, const uint8_t* in, cudaStream_t s, Launches& L) {
  uint32_t* word = h->d_status + 2;
  cudaMemsetAsync(word, 0, sizeof(uint32_t), s);
  anchor_coverage(h->comp, h->n, reinterpret_cast<const int32_t*>(in + 64), h->n_c, h->is_anchor,
                  word, s, L);
  cudaMemcpyAsync(h->h_status + 2, word, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
}

// after the stream of enqueue_anchor_check has been synchronised
static mesh_codec_status_t anchor_check_result(const mesh_codec* h) {
  return (h->h_status[2] & ST_NO_ANCHOR) ? MC_E_NO_ANCHOR_IN_COMPONENT : MC_OK;
}

static mesh_codec_status_t enqueue_decode(mesh_codec* h, const uint8_t* in, double* out,
                                          cudaStream_t s, Launches& L,
                                          const double* x0 = nullptr,
                                          const double* dict_ref = nullptr,
                                          const EncodeLayout* lay = nullptr) {
  enqueue_anchor_check(h, in, s, L);
  MC_TRY(cudaStreamSynchronize(s));
  MC_TRY(cudaGetLastError());
  const mesh_codec_status_t cov = anchor_check_result(h);
  if (cov != MC_OK) return cov;
  decode_prepare(h, in, s, L, x0, dict_ref, lay);
  if (h->dec.refine) {
    const mesh_codec_status_t st = decode_refine(h, s, L);
    if (st != MC_OK) return st;
  } else {
    while (decode_cg_chunk(h, 32, s, L)) {
      MC_TRY(cudaStreamSynchronize(s));
      if (*h->h_active == 0) break;
    }
  }
  decode_finish(h, out, s, L);
  return MC_OK;
}

__global__ void k_flag_not_converged(const int32_t* done, int W, uint32_t* status) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < W; c += gridDim.x * blockDim.x)
    if (done[c] != 1) atomicOr(status, ST_NOT_CONVERGED);
}

mesh_codec_status_t mesh_codec_decode(mesh_codec_t* h, const uint8_t* bitstream, size_t bytes,
                                      double* positions_out, void* stream) {
  return mesh_codec_decode_ex(h, bitstream, bytes, nullptr, positions_out, stream);
}

mesh_codec_status_t mesh_codec_decode_ex(mesh_codec_t* h, const uint8_t* bitstream, size_t bytes,
                                         const double* x0, double* positions_out, void* stream) {
  if (!h || !bitstream || !positions_out) return MC_E_INVALID_ARG;
  if (x0 && (((uintptr_t)x0 & 7) || use_factored(h))) return MC_E_INVALID_ARG;
  if (((uintptr_t)bitstream & 7) || ((uintptr_t)positions_out & 7)) return MC_E_INVALID_ARG;
  if (bytes < 64) return MC_E_BITSTREAM_CORRUPT;
  if (h->n_c == 0) return MC_E_INVALID_ARG;   // Eq. 12 needs anchors (L is singular)
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  MC_TRY(cudaMemcpyAsync(h->h_header, bitstream, 64, cudaMemcpyDeviceToHost, s));
  MC_TRY(cudaStreamSynchronize(s));
  mesh_codec_status_t st = check_header(h, h->h_header, bytes);
  if (st != MC_OK) return st;
  h->launches_decode = 0;
  Launches L{&h->launches_decode};
  st = enqueue_decode(h, bitstream, positions_out, s, L, x0);
  if (st != MC_OK) return st;
  MC_TRY(cudaGetLastError());
  st = read_status(h, s);
  settle_anchor_cache(h, st);
  prof_collect(h);
  return st;
}

mesh_codec_status_t mesh_codec_decode_stage(mesh_codec_t* h, const uint8_t* bitstream,
                                            size_t bytes, double* delta_out, double* anchors_out,
                                            void* stream) {
  if (!h || !bitstream) return MC_E_INVALID_ARG;
  if (((uintptr_t)bitstream & 7) || ((uintptr_t)delta_out & 7) || ((uintptr_t)anchors_out & 7))
    return MC_E_INVALID_ARG;
  if (bytes < 64) return MC_E_BITSTREAM_CORRUPT;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  MC_TRY(cudaMemcpyAsync(h->h_header, bitstream, 64, cudaMemcpyDeviceToHost, s));
  MC_TRY(cudaStreamSynchronize(s));
  mesh_codec_status_t st = check_header(h, h->h_header, bytes);
  if (st != MC_OK) return st;
  const int n = h->n, F = h->F, k = h->k, W = h->W;
  h->launches_decode = 0;
  Launches L{&h->launches_decode};
  cudaMemsetAsync(h->d_status, 0, sizeof(uint32_t), s);
  unpack_sections(bitstream, h->lay, h->Udeq, h->Cdeq, h->Ahat, h->dec_anchors, nullptr,
                  h->d_status, s, L);
  if (delta_out) {
    if (h->lp >= 0 && h->p.refine == 0) {
      mixed_backproject(h, s, L);
    } else {
      dgemm(n, F, k, 3, Strided{h->Cdeq, 1, n, (long long)k * n},
            Strided{h->Udeq, 1, k, (long long)F * k}, StridedOut{h->D, W, 1, F}, 1, nullptr, s,
            L);
    }
    MC_TRY(cudaMemcpyAsync(delta_out, h->D, sizeof(double) * n * W, cudaMemcpyDeviceToDevice, s));
  }
  if (anchors_out && h->n_c > 0)
    MC_TRY(cudaMemcpyAsync(anchors_out, h->Ahat, sizeof(double) * 3 * h->n_c * F,
                           cudaMemcpyDeviceToDevice, s));
  MC_TRY(cudaGetLastError());
  return read_status(h, s);
}

mesh_codec_status_t mesh_codec_set_start_basis(mesh_codec_t* h, const double* q0, void* stream) {
  if (!h) return MC_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  Launches L{&h->launches_create};
  MC_TRY(cudaMemsetAsync(h->d_status, 0, sizeof(uint32_t), s));
  if (q0) {
    MC_TRY(cudaMemcpyAsync(h->Q0, q0, sizeof(double) * 3 * h->F * h->k, cudaMemcpyDeviceToDevice,
                           s));
  } else {
    gen_start_basis(h->Q0, h->F, h->k, h->p.seed, s, L);
  }
  const int sg = gemm_splits(h->F, ((h->k + 63) / 64) * ((h->k + 31) / 32));
  cholqr3(h->Q0, h->F, h->k, qr_work(h, sg), nullptr, h->d_status, s, L);
  MC_TRY(cudaGetLastError());
  return read_status(h, s);
}

// ------------------------------------------------------------ blocks variant
static constexpr uint32_t kBlocksMagic = 0x42434D44u;   // "DMCB"

struct BlocksSizes {
  unsigned long long first, other, total;
};

static BlocksSizes blocks_sizes(const mesh_codec* h, int n_blocks) {
  BlocksSizes z;
  z.first = (unsigned long long)h->lay.total;
  z.other = (unsigned long long)(h->p.block_delta ? h->lay_delta.total : h->lay.total);
  z.total = 64ull + z.first + (unsigned long long)(n_blocks - 1) * z.other;
  return z;
}

mesh_codec_status_t mesh_codec_blocks_size(const mesh_codec_t* h, int n_blocks, size_t* bytes) {
  if (!h || !bytes || n_blocks < 1) return MC_E_INVALID_ARG;
  *bytes = (size_t)blocks_sizes(h, n_blocks).total;
  return MC_OK;
}

mesh_codec_status_t mesh_codec_rates(const mesh_codec_params_t* p, int n_blocks, double* out) {
  if (!out || n_blocks < 1 || !valid_params(p)) return MC_E_INVALID_ARG;
  const double n = p->n_vertices, F = p->n_frames, k = p->rank, nc = p->n_anchors;
  auto bits = [](int b) { return b == 0 ? 64.0 : (double)b; };
  const bool delta = p->block_delta != 0;
  const double db_first = bits(p->dict_bits);
  const double db_other = delta ? bits(p->block_delta_bits) : db_first;
  out[0] = bits(p->coeff_bits) * k / F;
  out[1] = bits(p->anchor_bits) * nc / n;
  out[2] = (db_first + (n_blocks - 1) * db_other) * k / (n * n_blocks);
  out[3] = out[0] + out[1] + out[2];
  const EncodeLayout first = make_layout(p->n_vertices, p->n_frames, p->rank, p->n_anchors,
                                         p->coeff_bits, p->dict_bits, p->anchor_bits,
                                         p->laplacian_kind);
  const EncodeLayout other = make_layout(p->n_vertices, p->n_frames, p->rank, p->n_anchors,
                                         p->coeff_bits,
                                         delta ? p->block_delta_bits : p->dict_bits,
                                         p->anchor_bits, p->laplacian_kind);
  const double bytes = n_blocks == 1
                           ? (double)first.total
                           : 64.0 + (double)first.total + (n_blocks - 1.0) * (double)other.total;
  out[4] = bytes * 8.0 / (n * F * n_blocks);
  return MC_OK;
}

mesh_codec_status_t mesh_codec_encode_blocks(mesh_codec_t* h, const double* positions,
                                             int n_blocks, uint8_t* out, size_t capacity,
                                             size_t* written, void* stream) {
  if (!h || !positions || !out || !written || n_blocks < 1) return MC_E_INVALID_ARG;
  if (((uintptr_t)out & 7) || ((uintptr_t)positions & 7)) return MC_E_INVALID_ARG;
  if (h->p.layout != MC_LAYOUT_FRAMES) return MC_E_INVALID_ARG;   // blocks are frame ranges
  const BlocksSizes z = blocks_sizes(h, n_blocks);
  *written = (size_t)z.total;
  if (capacity < z.total) return MC_E_BUFFER_TOO_SMALL;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  h->launches_encode = 0;
  Launches L{&h->launches_encode};
  const int n = h->n, F = h->F, k = h->k;
  const bool delta = h->p.block_delta != 0;
  const size_t basis_bytes = sizeof(double) * 3 * F * k;
  // container header, staged in pinned memory (read_status below waits for the copy)
  std::memset(h->h_header, 0, 64);
  const uint32_t w[5] = {kBlocksMagic, 1u, (uint32_t)n_blocks, delta ? 1u : 0u,
                         delta ? (uint32_t)h->p.block_delta_bits : 0u};
  const unsigned long long q[3] = {z.first, z.other, z.total};
  std::memcpy(h->h_header, w, sizeof(w));
  std::memcpy(h->h_header + sizeof(w), q, sizeof(q));
  MC_TRY(cudaMemcpyAsync(out, h->h_header, 64, cudaMemcpyHostToDevice, s));
  size_t off = 64;
  for (int b = 0; b < n_blocks; ++b) {
    const double* pos_b = positions + (size_t)b * F * n * 3;
    uint8_t* out_b = out + off;
    const bool dref = delta && b > 0;
    EncodeOpts o;
    if (b == 0) o.direct = F <= kDirectMaxFrames;   // Algorithm 1's SVD of R[1]
    else o.start = h->Ublk;                          // U[i]^(1) = U[i-1]
    if (dref) {
      o.dict_ref = h->Uhat;
      o.lay = &h->lay_delta;
    }
    enqueue_encode(h, pos_b, out_b, s, L, false, o);
    MC_TRY(cudaGetLastError());
    mesh_codec_status_t st = read_status(h, s);
    if (st != MC_OK) return st;
    MC_TRY(cudaMemcpyAsync(h->Ublk, h->U, basis_bytes, cudaMemcpyDeviceToDevice, s));
    if (delta) {
      // the dictionary the decoder will hold after this block (closed loop)
      unpack_sections(out_b, dref ? h->lay_delta : h->lay, h->Udeq, h->Cdeq, h->Ahat,
                      h->dec_anchors, nullptr, h->d_status, s, L);
      if (dref) {
        const long long cnt = 3LL * F * k;
        k_axpy_sub<<<(int)std::min<long long>((cnt + 255) / 256, 1024), 256, 0, s>>>(
            h->Udeq, h->Uhat, cnt, 1.0, h->Uhat);
        L.add(1);
      } else {
        MC_TRY(cudaMemcpyAsync(h->Uhat, h->Udeq, basis_bytes, cudaMemcpyDeviceToDevice, s));
      }
    }
    off += (size_t)(b == 0 ? z.first : z.other);
  }
  MC_TRY(cudaGetLastError());
  return read_status(h, s);
}

mesh_codec_status_t mesh_codec_decode_blocks(mesh_codec_t* h, const uint8_t* in, size_t bytes,
                                             double* positions_out, void* stream) {
  if (!h || !in || !positions_out) return MC_E_INVALID_ARG;
  if (((uintptr_t)in & 7) || ((uintptr_t)positions_out & 7)) return MC_E_INVALID_ARG;
  if (h->p.layout != MC_LAYOUT_FRAMES) return MC_E_INVALID_ARG;   // blocks are frame ranges
  if (bytes < 64) return MC_E_BITSTREAM_CORRUPT;
  if (h->n_c == 0) return MC_E_INVALID_ARG;   // Eq. 12 needs anchors
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  MC_TRY(cudaMemcpyAsync(h->h_header, in, 64, cudaMemcpyDeviceToHost, s));
  MC_TRY(cudaStreamSynchronize(s));
  uint32_t w[5];
  unsigned long long q[3];
  std::memcpy(w, h->h_header, sizeof(w));
  std::memcpy(q, h->h_header + sizeof(w), sizeof(q));
  if (w[0] != kBlocksMagic || w[1] != 1u || w[2] < 1u || w[2] > (1u << 24) || (w[3] & ~1u))
    return MC_E_BITSTREAM_CORRUPT;
  const int n_blocks = (int)w[2];
  const bool delta = (w[3] & 1u) != 0;
  if (delta != (h->p.block_delta != 0) || (delta && (int)w[4] != h->p.block_delta_bits))
    return MC_E_BITSTREAM_CORRUPT;
  const BlocksSizes z = blocks_sizes(h, n_blocks);
  if (q[0] != z.first || q[1] != z.other || q[2] != z.total || bytes != (size_t)z.total)
    return MC_E_BITSTREAM_CORRUPT;
  const int n = h->n, F = h->F, k = h->k;
  const bool frames = !use_factored(h);
  h->launches_decode = 0;
  Launches L{&h->launches_decode};
  mesh_codec_status_t worst = MC_OK;
  size_t off = 64;
  for (int b = 0; b < n_blocks; ++b) {
    const uint8_t* in_b = in + off;
    const size_t nbytes = (size_t)(b == 0 ? z.first : z.other);
    const bool dref = delta && b > 0;
    const EncodeLayout* lay = dref ? &h->lay_delta : &h->lay;
    MC_TRY(cudaMemcpyAsync(h->h_header, in_b, 64, cudaMemcpyDeviceToHost, s));
    MC_TRY(cudaStreamSynchronize(s));
    mesh_codec_status_t st = check_header(h, h->h_header, nbytes, lay);
    if (st != MC_OK) return st;
    double* out_b = positions_out + (size_t)b * F * n * 3;
    const double* x0 = nullptr;
    if (frames && b > 0) {
      // the previous block's last decoded frame, repeated, as the first iterate
      // (R is free until the CG starts)
      st = mesh_codec_warm_compose(n, F, out_b - (size_t)n * 3, nullptr, h->R, s);
      if (st != MC_OK) return st;
      L.add(1);
      x0 = h->R;
    }
    st = enqueue_decode(h, in_b, out_b, s, L, x0, dref ? h->Uhat : nullptr, lay);
    if (st != MC_OK) return st;
    MC_TRY(cudaGetLastError());
    st = read_status(h, s);
    settle_anchor_cache(h, st);
    if (st == MC_E_NOT_CONVERGED) worst = st;
    else if (st != MC_OK) return st;
    if (delta)
      MC_TRY(cudaMemcpyAsync(h->Uhat, h->Udeq, sizeof(double) * 3 * F * k,
                             cudaMemcpyDeviceToDevice, s));
    off += nbytes;
  }
  MC_TRY(cudaStreamSynchronize(s));
  prof_collect(h);
  return worst;
}

static mesh_codec_status_t ensure_staging(mesh_codec* h) {
  if (!h->stage_pos) MC_TRY(cudaMalloc(&h->stage_pos, sizeof(double) * 3ull * h->n * h->F));
  if (!h->stage_bits) MC_TRY(cudaMalloc(&h->stage_bits, (size_t)h->lay.total));
  return MC_OK;
}

mesh_codec_status_t mesh_codec_encode_host(mesh_codec_t* h, const double* positions_host,
                                           uint8_t* bitstream_host, size_t capacity,
                                           size_t* written, void* stream) {
  if (!h || !positions_host || !bitstream_host || !written) return MC_E_INVALID_ARG;
  *written = (size_t)h->lay.total;
  if (capacity < (size_t)h->lay.total) return MC_E_BUFFER_TOO_SMALL;
  mesh_codec_status_t st = ensure_staging(h);
  if (st != MC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  MC_TRY(cudaMemcpyAsync(h->stage_pos, positions_host, sizeof(double) * 3ull * h->n * h->F,
                         cudaMemcpyHostToDevice, s));
  h->launches_encode = 0;
  Launches L{&h->launches_encode};
  enqueue_encode(h, h->stage_pos, h->stage_bits, s, L, true);
  MC_TRY(cudaMemcpyAsync(bitstream_host, h->stage_bits, (size_t)h->lay.total,
                         cudaMemcpyDeviceToHost, s));
  MC_TRY(cudaGetLastError());
  return read_status(h, s);
}

mesh_codec_status_t mesh_codec_decode_host(mesh_codec_t* h, const uint8_t* bitstream_host,
                                           size_t bytes, double* positions_out_host, void* stream) {
  if (!h || !bitstream_host || !positions_out_host) return MC_E_INVALID_ARG;
  if (bytes < 64) return MC_E_BITSTREAM_CORRUPT;
  if (h->n_c == 0) return MC_E_INVALID_ARG;
  mesh_codec_status_t st = check_header(h, bitstream_host, bytes);
  if (st != MC_OK) return st;
  st = ensure_staging(h);
  if (st != MC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  MC_TRY(cudaMemcpyAsync(h->stage_bits, bitstream_host, bytes, cudaMemcpyHostToDevice, s));
  h->launches_decode = 0;
  Launches L{&h->launches_decode};
  st = enqueue_decode(h, h->stage_bits, h->stage_pos, s, L);
  if (st != MC_OK) return st;
  MC_TRY(cudaMemcpyAsync(positions_out_host, h->stage_pos, sizeof(double) * 3ull * h->n * h->F,
                         cudaMemcpyDeviceToHost, s));
  MC_TRY(cudaGetLastError());
  st = read_status(h, s);
  settle_anchor_cache(h, st);
  prof_collect(h);
  return st;
}

// ------------------------------------------------------------ batches
// Grouped CG of a batch (mesh_codec_decode_batch): the FP32 solves whose
// column count is a multiple of 4 advance together, each phase of an
// iteration one launch over a work table of (solve, row block, column tile)
// items and (solve, column) items, one CTA per item; the
// table lives in device memory, so one captured graph of 32 iterations
// serves the whole decode while finished solves leave the table between
// runs.  Every solve keeps its own geometry, vectors and reduction order,
// so its result equals the result of decoding it alone.
__global__ void k_gather_active(const CgSeq* __restrict__ seqs, int n, int32_t* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = *seqs[i].active;
}

struct GroupedCg {
  std::vector<mesh_codec*> hs;   // the grouped handles, in table order
  std::vector<char> live;        // per solve: still iterating
  char* dbuf = nullptr;          // device: solves, row items, column items, counts, active
  char* hbuf = nullptr;          // pinned: table staging and the active counts
  CgSeq* d_seqs = nullptr;
  int4* d_items = nullptr;
  int2* d_cols = nullptr;
  int* d_counts = nullptr;       // [0] row items, [1] column items
  int32_t* d_act = nullptr;
  CgSeq* h_seqs = nullptr;
  int4* h_items = nullptr;
  int2* h_cols = nullptr;
  int* h_counts = nullptr;
  int32_t* h_act = nullptr;
  int grid_rows = 0, grid_cols = 0;
  size_t smem = 0;
  cudaStream_t s = nullptr;      // the grouped solves' stream
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev = nullptr;

  ~GroupedCg() {
    if (exec) cudaGraphExecDestroy(exec);
    if (ev) cudaEventDestroy(ev);
    if (dbuf) cudaFree(dbuf);
    if (hbuf) cudaFreeHost(hbuf);
  }
  bool any_live() const {
    for (char l : live)
      if (l) return true;
    return false;
  }
  // rebuild the tables of the live solves into pinned memory and upload them on s
  cudaError_t upload_tables() {
    int ni = 0, nc = 0;
    for (size_t q = 0; q < hs.size(); ++q) {
      if (!live[q]) continue;
      const CgGeom& g = h_seqs[q].g;
      const int tiles = (g.W + kGroupCols - 1) / kGroupCols;
      for (int by = 0; by < g.row_blocks; ++by)
        for (int bx = 0; bx < tiles; ++bx) h_items[ni++] = make_int4((int)q, by, bx, 0);
      for (int c = 0; c < g.W; ++c) h_cols[nc++] = make_int2((int)q, c);
    }
    h_counts[0] = ni;
    h_counts[1] = nc;
    cudaError_t e = cudaMemcpyAsync(d_items, h_items, sizeof(int4) * std::max(ni, 1),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_cols, h_cols, sizeof(int2) * std::max(nc, 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_counts, h_counts, sizeof(int) * 2, cudaMemcpyHostToDevice, s);
    return e;
  }
};

// set up the grouped solves of `hs` (phase 1 done on their own streams)
static mesh_codec_status_t grouped_setup(GroupedCg& G) {
  const size_t S = G.hs.size();
  size_t max_items = 0, max_cols = 0;
  for (mesh_codec* h : G.hs) {
    const CgGeom& g = h->dec.geom;
    max_items += (size_t)g.row_blocks * ((g.W + kGroupCols - 1) / kGroupCols);
    max_cols += (size_t)g.W;
    G.smem = std::max(G.smem, cg4_grouped_smem(g));
  }
  auto carve = [](size_t& off, size_t bytes) {
    off = (off + 255) & ~size_t(255);
    const size_t at = off;
    off += std::max<size_t>(bytes, 1);
    return at;
  };
  size_t off = 0;
  const size_t o_seqs = carve(off, sizeof(CgSeq) * S), o_items = carve(off, sizeof(int4) * max_items);
  const size_t o_cols = carve(off, sizeof(int2) * max_cols), o_counts = carve(off, sizeof(int) * 2);
  const size_t o_act = carve(off, sizeof(int32_t) * S);
  MC_TRY(cudaMalloc(&G.dbuf, off));
  MC_TRY(cudaMallocHost(&G.hbuf, off));
  G.d_seqs = (CgSeq*)(G.dbuf + o_seqs);   G.h_seqs = (CgSeq*)(G.hbuf + o_seqs);
  G.d_items = (int4*)(G.dbuf + o_items);  G.h_items = (int4*)(G.hbuf + o_items);
  G.d_cols = (int2*)(G.dbuf + o_cols);    G.h_cols = (int2*)(G.hbuf + o_cols);
  G.d_counts = (int*)(G.dbuf + o_counts); G.h_counts = (int*)(G.hbuf + o_counts);
  G.d_act = (int32_t*)(G.dbuf + o_act);   G.h_act = (int32_t*)(G.hbuf + o_act);
  for (size_t q = 0; q < S; ++q) {
    mesh_codec* h = G.hs[q];
    const DecodeState& d = h->dec;
    CgSeq& c = G.h_seqs[q];
    c.g = d.geom;
    c.row_ptr = h->row_ptr; c.col_idx = h->col_idx; c.deg = h->deg;
    c.inv_d = (const float*)d.inv_d; c.inv_diag = (const float*)d.inv_diag;
    c.is_anchor = h->is_anchor;
    c.X = (float*)h->X; c.R = (float*)h->R; c.P = (float*)h->P; c.T = (float*)h->Tv;
    c.Q = (float*)h->Qv;
    c.partials = h->cg.partials; c.rz = h->cg.rz; c.rr = h->cg.rr; c.bb = h->cg.bb;
    c.alpha = h->cg.alpha; c.beta = h->cg.beta;
    c.done = h->cg.done; c.iters = h->cg.iters; c.active = h->cg.active;
    c.kind = h->kind;
    c.max_iters = h->p.cg_max_iters;
    c.rtol2 = h->p.cg_rtol * h->p.cg_rtol;
  }
  G.live.assign(S, 1);
  G.s = G.hs[0]->own;
  MC_TRY(cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming));
  // the grouped stream waits for every solve's phase 1
  for (size_t q = 1; q < S; ++q) {
    MC_TRY(cudaEventRecord(G.hs[q]->ev_chunk, G.hs[q]->own));
    MC_TRY(cudaStreamWaitEvent(G.s, G.hs[q]->ev_chunk, 0));
  }
  MC_TRY(cudaMemcpyAsync(G.d_seqs, G.h_seqs, sizeof(CgSeq) * S, cudaMemcpyHostToDevice, G.s));
  MC_TRY(G.upload_tables());
  // one CTA per item of the full table (CTAs past the shrinking table return)
  G.grid_rows = (int)std::max<size_t>(1, max_items);
  G.grid_cols = (int)std::max<size_t>(1, max_cols);
  // one graph: 32 iterations, then every solve's active-column count to pinned memory
  cudaStream_t cap = G.hs[0]->cap;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MC_E_CUDA;
  Launches none{nullptr};
  for (int j = 0; j < kCgChunk; ++j)
    cg4_grouped_iteration(G.d_seqs, G.d_items, G.d_counts, G.d_cols, G.d_counts + 1, G.grid_rows,
                          G.grid_cols, G.smem, cap, none);
  k_gather_active<<<1, 256, 0, cap>>>(G.d_seqs, (int)S, G.d_act);
  cudaMemcpyAsync(G.h_act, G.d_act, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, cap);
  cudaGraph_t graph = nullptr;
  if (cudaStreamEndCapture(cap, &graph) != cudaSuccess || !graph) {
    cudaGetLastError();
    return MC_E_CUDA;
  }
  const cudaError_t e = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    G.exec = nullptr;
    return MC_E_CUDA;
  }
  return MC_OK;
}

// one run of 32 grouped iterations, enqueued on the grouped stream
static mesh_codec_status_t grouped_run(GroupedCg& G) {
  MC_TRY(cudaGraphLaunch(G.exec, G.s));
  for (size_t q = 0; q < G.hs.size(); ++q)
    if (G.live[q]) G.hs[q]->launches_decode += 6 * kCgChunk;
  MC_TRY(cudaEventRecord(G.ev, G.s));
  return MC_OK;
}

// after the run's event: count its iterations, retire finished solves
static mesh_codec_status_t grouped_retire(GroupedCg& G) {
  bool changed = false;
  for (size_t q = 0; q < G.hs.size(); ++q) {
    if (!G.live[q]) continue;
    mesh_codec* h = G.hs[q];
    h->dec.it = std::min(h->dec.it + kCgChunk, h->p.cg_max_iters);
    if (G.h_act[q] == 0 || h->dec.it >= h->p.cg_max_iters) {
      G.live[q] = 0;
      changed = true;
    }
  }
  if (changed && G.any_live()) MC_TRY(G.upload_tables());
  return MC_OK;
}

// Each handle runs on its own stream, forked from and joined back to the
// caller's stream with events, so independent sequences of uneven sizes
// overlap on the GPU.
static bool batch_args_ok(mesh_codec_t* const* hs, int count) {
  if (!hs || count < 1) return false;
  for (int i = 0; i < count; ++i)
    if (!hs[i]) return false;
  for (int i = 0; i < count; ++i)
    for (int j = i + 1; j < count; ++j)
      if (hs[i] == hs[j]) return false;   // a handle's workspace is used once per batch
  return true;
}

mesh_codec_status_t mesh_codec_encode_batch(mesh_codec_t* const* handles, int count,
                                            const double* const* positions,
                                            uint8_t* const* bitstreams,
                                            const size_t* capacities, size_t* written,
                                            mesh_codec_status_t* statuses, void* stream) {
  if (!batch_args_ok(handles, count) || !positions || !bitstreams || !capacities || !written)
    return MC_E_INVALID_ARG;
  cudaStream_t s0 = (cudaStream_t)stream;
  MC_TRY(cudaEventRecord(handles[0]->ev_fork, s0));
  std::vector<mesh_codec_status_t> st(count, MC_OK);
  for (int i = 0; i < count; ++i) {
    mesh_codec* h = handles[i];
    written[i] = (size_t)h->lay.total;
    if (!positions[i] || !bitstreams[i] || ((uintptr_t)bitstreams[i] & 7)) {
      st[i] = MC_E_INVALID_ARG;
      continue;
    }
    if (capacities[i] < (size_t)h->lay.total) {
      st[i] = MC_E_BUFFER_TOO_SMALL;
      continue;
    }
    MC_TRY(cudaStreamWaitEvent(h->own, handles[0]->ev_fork, 0));
    h->last_stream = h->own;
    h->launches_encode = 0;
    Launches L{&h->launches_encode};
    enqueue_encode(h, positions[i], bitstreams[i], h->own, L, false);
    MC_TRY(cudaEventRecord(h->ev_done, h->own));
    MC_TRY(cudaStreamWaitEvent(s0, h->ev_done, 0));
  }
  mesh_codec_status_t first = MC_OK;
  for (int i = 0; i < count; ++i) {
    if (st[i] == MC_OK) st[i] = read_status(handles[i], handles[i]->own);
    if (statuses) statuses[i] = st[i];
    if (first == MC_OK) first = st[i];
  }
  return first;
}

mesh_codec_status_t mesh_codec_decode_batch(mesh_codec_t* const* handles, int count,
                                            const uint8_t* const* bitstreams,
                                            const size_t* bytes, double* const* positions_out,
                                            mesh_codec_status_t* statuses, void* stream) {
  return mesh_codec_decode_batch_ex(handles, count, bitstreams, bytes, positions_out, statuses,
                                    0, stream);
}

mesh_codec_status_t mesh_codec_decode_batch_ex(mesh_codec_t* const* handles, int count,
                                               const uint8_t* const* bitstreams,
                                               const size_t* bytes, double* const* positions_out,
                                               mesh_codec_status_t* statuses, int flags,
                                               void* stream) {
  if (!batch_args_ok(handles, count) || !bitstreams || !bytes || !positions_out)
    return MC_E_INVALID_ARG;
  if (flags & ~MC_BATCH_GROUPED) return MC_E_INVALID_ARG;
  cudaStream_t s0 = (cudaStream_t)stream;
  MC_TRY(cudaEventRecord(handles[0]->ev_fork, s0));
  std::vector<mesh_codec_status_t> st(count, MC_OK);
  // headers, all at once
  for (int i = 0; i < count; ++i) {
    mesh_codec* h = handles[i];
    if (!bitstreams[i] || !positions_out[i] || ((uintptr_t)bitstreams[i] & 7) ||
        ((uintptr_t)positions_out[i] & 7) || h->n_c == 0) {
      st[i] = MC_E_INVALID_ARG;
      continue;
    }
    if (bytes[i] < 64) {
      st[i] = MC_E_BITSTREAM_CORRUPT;
      continue;
    }
    MC_TRY(cudaStreamWaitEvent(h->own, handles[0]->ev_fork, 0));
    MC_TRY(cudaMemcpyAsync(h->h_header, bitstreams[i], 64, cudaMemcpyDeviceToHost, h->own));
  }
  for (int i = 0; i < count; ++i) {
    if (st[i] != MC_OK) continue;
    MC_TRY(cudaStreamSynchronize(handles[i]->own));
    st[i] = check_header(handles[i], handles[i]->h_header, bytes[i]);
  }
  // every stream's anchors cover every component of its mesh (Eq. 12)
  for (int i = 0; i < count; ++i) {
    if (st[i] != MC_OK) continue;
    mesh_codec* h = handles[i];
    h->launches_decode = 0;
    Launches L{&h->launches_decode};
    enqueue_anchor_check(h, bitstreams[i], h->own, L);
  }
  for (int i = 0; i < count; ++i) {
    if (st[i] != MC_OK) continue;
    MC_TRY(cudaStreamSynchronize(handles[i]->own));
    st[i] = anchor_check_result(handles[i]);
  }
  // phase 1 for every sequence, then their CG solves in lockstep chunks
  std::vector<int> active;
  for (int i = 0; i < count; ++i) {
    if (st[i] != MC_OK) continue;
    mesh_codec* h = handles[i];
    h->last_stream = h->own;
    Launches L{&h->launches_decode};
    decode_prepare(h, bitstreams[i], h->own, L);
    if (h->dec.refine) {
      // refined solves synchronise per outer step: run them one by one
      st[i] = decode_refine(h, h->own, L);
      continue;
    }
    active.push_back(i);
  }
  // with MC_BATCH_GROUPED the FP32 solves with a multiple of 4 columns advance
  // as grouped batches; the others (FP64, frames solves of 3F % 4 != 0
  // columns, kernel timing) run their own chunks on their own streams alongside
  // The candidates are dealt, largest first, over up to kGroups grouped
  // batches on streams of their own, so that different phases of different
  // batches (latency-bound gathers, bandwidth-bound updates) overlap.
  constexpr int kGroups = 4;
  std::vector<mesh_codec*> cand;
  std::vector<int> alone;
  for (int i : active) {
    mesh_codec* h = handles[i];
    if (h->dec.single && !h->dec.refine && h->dec.Wc % 4 == 0 && h->prof_every == 0)
      cand.push_back(h);
    else
      alone.push_back(i);
  }
  std::vector<std::unique_ptr<GroupedCg>> groups;
  if (cand.size() < 2 || !(flags & MC_BATCH_GROUPED)) {
    alone = active;
  } else {
    std::stable_sort(cand.begin(), cand.end(), [](const mesh_codec* a, const mesh_codec* b) {
      return (long long)a->n * a->dec.Wc > (long long)b->n * b->dec.Wc;
    });
    const int ng = std::max(1, std::min<int>(kGroups, (int)cand.size() / 2));
    for (int g = 0; g < ng; ++g) groups.emplace_back(new GroupedCg());
    for (size_t q = 0; q < cand.size(); ++q) groups[q % ng]->hs.push_back(cand[q]);
    for (auto& G : groups) {
      const mesh_codec_status_t gs = grouped_setup(*G);
      if (gs != MC_OK) return gs;
    }
  }
  auto any_group_live = [&]() {
    for (auto& G : groups)
      if (G->any_live()) return true;
    return false;
  };
  while (!alone.empty() || any_group_live()) {
    std::vector<int> issued;
    for (int i : alone) {
      mesh_codec* h = handles[i];
      Launches L{&h->launches_decode};
      if (decode_cg_chunk(h, 32, h->own, L)) {
        MC_TRY(cudaEventRecord(h->ev_chunk, h->own));
        issued.push_back(i);
      }
    }
    std::vector<GroupedCg*> ran;
    for (auto& G : groups) {
      if (!G->any_live()) continue;
      const mesh_codec_status_t gs = grouped_run(*G);
      if (gs != MC_OK) return gs;
      ran.push_back(G.get());
    }
    std::vector<int> still;
    for (int i : issued) {
      MC_TRY(cudaEventSynchronize(handles[i]->ev_chunk));
      if (*handles[i]->h_active != 0) still.push_back(i);
    }
    alone.swap(still);
    for (GroupedCg* G : ran) {
      MC_TRY(cudaEventSynchronize(G->ev));
      const mesh_codec_status_t gs = grouped_retire(*G);
      if (gs != MC_OK) return gs;
    }
  }
  for (auto& G : groups) {
    // every grouped handle's stream continues after its grouped solves
    MC_TRY(cudaEventRecord(G->ev, G->s));
    for (mesh_codec* h : G->hs) MC_TRY(cudaStreamWaitEvent(h->own, G->ev, 0));
  }
  for (int i = 0; i < count; ++i) {
    if (st[i] != MC_OK) continue;
    mesh_codec* h = handles[i];
    Launches L{&h->launches_decode};
    decode_finish(h, positions_out[i], h->own, L);
    MC_TRY(cudaEventRecord(h->ev_done, h->own));
    MC_TRY(cudaStreamWaitEvent(s0, h->ev_done, 0));
  }
  mesh_codec_status_t first = MC_OK;
  for (int i = 0; i < count; ++i) {
    if (st[i] == MC_OK) {
      st[i] = read_status(handles[i], handles[i]->own);
      prof_collect(handles[i]);
    }
    settle_anchor_cache(handles[i], st[i]);
    if (statuses) statuses[i] = st[i];
    if (first == MC_OK) first = st[i];
  }
  return first;
}

mesh_codec_status_t mesh_codec_set_profiling(mesh_codec_t* h, int every) {
  if (!h || every < 0) return MC_E_INVALID_ARG;
  h->prof_every = every;
  h->prof_used = 0;
  h->run_used = 0;
  for (int k = 0; k < MESH_CODEC_PROF_KERNELS; ++k) {
    h->prof_ms[k] = 0.0;
    h->prof_launches[k] = 0;
  }
  return MC_OK;
}

mesh_codec_status_t mesh_codec_get_profile(const mesh_codec_t* hc, mesh_codec_profile_t* out) {
  if (!hc || !out) return MC_E_INVALID_ARG;
  mesh_codec* h = const_cast<mesh_codec*>(hc);
  MC_TRY(cudaStreamSynchronize(h->last_stream));
  std::memset(out, 0, sizeof(*out));
  out->n_kernels = kCgKernels + 1;
  for (int k = 0; k < kCgKernels; ++k) {
    std::snprintf(out->name[k], sizeof(out->name[k]), "%s", kCgKernelNames[k]);
    out->launches_timed[k] = h->prof_launches[k];
    out->total_ms[k] = h->prof_ms[k];
  }
  // whole iterations timed as runs (graph replays), without per-kernel events
  std::snprintf(out->name[kCgKernels], sizeof(out->name[kCgKernels]), "%s", "cg_iteration");
  out->launches_timed[kCgKernels] = h->prof_launches[kCgKernels];
  out->total_ms[kCgKernels] = h->prof_ms[kCgKernels];
  return MC_OK;
}

mesh_codec_status_t mesh_codec_get_stats(const mesh_codec_t* hc, mesh_codec_stats_t* st) {
  if (!hc || !st) return MC_E_INVALID_ARG;
  mesh_codec* h = const_cast<mesh_codec*>(hc);
  std::memset(st, 0, sizeof(*st));
  MC_TRY(cudaStreamSynchronize(h->last_stream));
  for (int c = 0; c < 3; ++c) {
    st->oi_sweeps[c] = h->oi_done[c];
    st->oi_change[c] = h->oi_last_change[c];
  }
  st->launches_create = h->launches_create;
  st->launches_encode = h->launches_encode;
  st->launches_decode = h->launches_decode;
  st->workspace_bytes = h->ws_bytes;
  if (h->cg_columns > 0) {
    std::vector<int32_t> it(h->cg_columns), dn(h->cg_columns);
    std::vector<double> rr(h->cg_columns), bb(h->cg_columns);
    MC_TRY(cudaMemcpy(it.data(), h->cg.iters, sizeof(int32_t) * it.size(), cudaMemcpyDeviceToHost));
    MC_TRY(cudaMemcpy(dn.data(), h->cg.done, sizeof(int32_t) * dn.size(), cudaMemcpyDeviceToHost));
    MC_TRY(cudaMemcpy(rr.data(), h->cg.rr, sizeof(double) * rr.size(), cudaMemcpyDeviceToHost));
    MC_TRY(cudaMemcpy(bb.data(), h->cg.bb, sizeof(double) * bb.size(), cudaMemcpyDeviceToHost));
    int mx = 0, mn = 1 << 30, nc = 0;
    double sum = 0.0, res = 0.0;
    for (int i = 0; i < h->cg_columns; ++i) {
      mx = std::max(mx, it[i]);
      mn = std::min(mn, it[i]);
      sum += it[i];
      if (dn[i] != 1) ++nc;
      if (bb[i] > 0.0 && it[i] > 0) res = std::max(res, std::sqrt(rr[i] / bb[i]));
    }
    st->cg_iters_max = mx;
    st->cg_iters_min = mn;
    st->cg_iters_mean = sum / h->cg_columns;
    st->cg_columns = h->cg_columns;
    st->cg_iterations_run = h->dec.it;
    st->cg_not_converged = nc;
    st->cg_rel_residual_max = res;
  }
  return MC_OK;
}

mesh_codec_status_t mesh_codec_buffer_size(const mesh_codec_t* h, int which, size_t* count,
                                           size_t* elem_bytes) {
  if (!h || !count || !elem_bytes) return MC_E_INVALID_ARG;
  const size_t n = h->n, F = h->F, k = h->k, W = h->W;
  switch (which) {
    case MC_BUF_ROW_PTR: *count = n + 1; *elem_bytes = 4; break;
    case MC_BUF_COL_IDX: *count = (size_t)h->nnz; *elem_bytes = 4; break;
    case MC_BUF_DEGREE: *count = n; *elem_bytes = 4; break;
    case MC_BUF_ANCHORS: *count = (size_t)h->n_c; *elem_bytes = 4; break;
    case MC_BUF_DELTA: *count = n * W; *elem_bytes = 8; break;
    case MC_BUF_BASIS: *count = 3 * F * k; *elem_bytes = 8; break;
    case MC_BUF_RITZ: *count = 3 * k; *elem_bytes = 8; break;
    case MC_BUF_COEFF: *count = 3 * k * n; *elem_bytes = 8; break;
    case MC_BUF_START: *count = 3 * F * k; *elem_bytes = 8; break;
    case MC_BUF_DELTA_REC: *count = n * W; *elem_bytes = 8; break;
    case MC_BUF_CG_ITERS: *count = (size_t)h->cg_columns; *elem_bytes = 4; break;
    default: return MC_E_INVALID_ARG;
  }
  return MC_OK;
}

mesh_codec_status_t mesh_codec_copy_buffer(const mesh_codec_t* h, int which, void* dst,
                                           size_t count, void* stream) {
  size_t cnt = 0, eb = 0;
  mesh_codec_status_t st = mesh_codec_buffer_size(h, which, &cnt, &eb);
  if (st != MC_OK) return st;
  if (!dst || count != cnt) return MC_E_INVALID_ARG;
  const void* src = nullptr;
  switch (which) {
    case MC_BUF_ROW_PTR: src = h->row_ptr; break;
    case MC_BUF_COL_IDX: src = h->col_idx; break;
    case MC_BUF_DEGREE: src = h->deg; break;
    case MC_BUF_ANCHORS: src = h->anchors; break;
    case MC_BUF_DELTA: src = h->D; break;
    case MC_BUF_BASIS: src = h->U; break;
    case MC_BUF_RITZ: src = h->theta; break;
    case MC_BUF_COEFF: src = h->Cf; break;
    case MC_BUF_START: src = h->Q0; break;
    case MC_BUF_DELTA_REC: src = h->D; break;
    case MC_BUF_CG_ITERS: src = h->cg.iters; break;
  }
  if (cnt == 0) return MC_OK;
  MC_TRY(cudaMemcpyAsync(dst, src, cnt * eb, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return MC_OK;
}

}  // extern "C"
