// Internal declarations shared by the codec's translation units.
//
// Device data layout (one handle, one connectivity):
//   vertex-major frame matrices  [n][W], W = 3F, column c*F + f holds
//   coordinate c of frame f; a vertex's whole trajectory (all three
//   coordinates) is one contiguous row, so the Laplacian's neighbour gathers
//   read contiguous rows and the per-coordinate matrix A_c^T (n x F) is a
//   strided view.
//   CSR adjacency without the diagonal (row_ptr [n+1], col_idx [nnz], deg [n]).
//   Small dense matrices per coordinate: [3][F][k] row-major.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/mesh_codec.h"

namespace mc {

// status bits set by device code (atomicOr into Handle::d_status)
enum : uint32_t {
  ST_BAD_INDEX = 1u << 0,
  ST_DEGENERATE = 1u << 1,
  ST_ISOLATED = 1u << 2,
  ST_CHOL_BREAKDOWN = 1u << 3,
  ST_BAD_ANCHORS = 1u << 4,
  ST_NOT_CONVERGED = 1u << 5,
  ST_BITSTREAM = 1u << 6,
  ST_TC_TIMEOUT = 1u << 7,   // a tensor-core GEMM wait ran out (bounded mbarrier wait)
  ST_NO_ANCHOR = 1u << 8,    // a connected component holds no anchor (Eq. 12 singular)
};

// splitmix64 (Steele, Lea, Flood 2014): output i of the generator seeded with s.
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t s, uint64_t i) {
  uint64_t z = s + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// The codec's salts: part of its definition ("anchors!", "basis_00").
constexpr uint64_t kAnchorSalt = 0x616E63686F727321ull;
constexpr uint64_t kBasisSalt = 0x62617369735F3030ull;
// completion of a numerically rank-deficient basis ("complete")
constexpr uint64_t kCompleteSalt = 0x636F6D706C657465ull;

struct Launches {
  uint64_t* counter = nullptr;
  void add(uint64_t k = 1) { if (counter) *counter += k; }
};

// ---------------------------------------------------------------- graph
struct CsrBuildTmp {
  int32_t* raw_deg;     // [n]
  int32_t* raw_off;     // [n+1]
  int32_t* cursor;      // [n]
  int32_t* raw_col;     // [6T]
  int32_t* scan_tmp;    // scan scratch
};
size_t scan_tmp_elems(int n);
void exclusive_scan_i32(const int32_t* in, int32_t* out, int n, int32_t* tmp,
                        cudaStream_t s, Launches& L);  // out has n+1 entries
void build_csr(const int32_t* tris, int T, int n, CsrBuildTmp& t, int32_t* row_ptr,
               int32_t* col_idx_or_null, int32_t* deg, uint32_t* status, cudaStream_t s,
               Launches& L);
void compact_csr(const CsrBuildTmp& t, const int32_t* row_ptr, int32_t* col_idx, int n,
                 cudaStream_t s, Launches& L);
void select_anchors(int n, int n_c, uint64_t seed, int32_t* anchors, cudaStream_t s,
                    Launches& L);
void check_anchors(const int32_t* anchors, int n_c, int n, uint32_t* status, cudaStream_t s,
                   Launches& L);
// comp[i] = smallest vertex index of i's connected component (parent: [n] scratch)
void component_labels(const int32_t* row_ptr, const int32_t* col_idx, int n, int32_t* parent,
                      int32_t* comp, cudaStream_t s, Launches& L);
// ST_NO_ANCHOR into *status when a component holds none of the n_c anchors
// (flag: [n] bytes of scratch)
void anchor_coverage(const int32_t* comp, int n, const int32_t* anchors, int n_c, uint8_t* flag,
                     uint32_t* status, cudaStream_t s, Launches& L);
void vertex_scalars_marked(const int32_t* row_ptr, const int32_t* col_idx, const int32_t* deg,
                           const uint8_t* is_anchor, int n, int kind, double* inv_d,
                           double* inv_diag_m, cudaStream_t s, Launches& L);
// delta = L X over W columns (Eq. 3 sum-then-divide / Eq. 4), bit-exact order
void laplacian_rows(const int32_t* row_ptr, const int32_t* col_idx, const int32_t* deg,
                    const double* X, double* Y, int n, int W, int kind, cudaStream_t s,
                    Launches& L);
// B = L^T Y (+ anchors scattered by a separate call)
void laplacian_t_rows(const int32_t* row_ptr, const int32_t* col_idx, const int32_t* deg,
                      const double* inv_d, const double* Y, double* B, int n, int W, int kind,
                      cudaStream_t s, Launches& L);

// ---------------------------------------------------------------- layout
void frames_to_vertex_major(const double* pos, double* X, int F, int n, cudaStream_t s,
                            Launches& L);
void vertex_major_to_frames(const double* X, double* pos, int F, int n, cudaStream_t s,
                            Launches& L);

// ---------------------------------------------------------------- dense FP64
struct Strided {  // element (r, c) at p[r*s0 + c*s1] + batch*sb
  const double* p;
  long long s0, s1, sb;
};
struct StridedOut {
  double* p;
  long long s0, s1, sb;
  int accumulate = 0;   // 1: C += A B
};
// C(b) = A(b) B(b) for b < batch, (M x K)(K x N); split-K into `splits` partial
// sums reduced in fixed order (partials: splits*batch*M*N doubles)
void dgemm(int M, int N, int K, int batch, Strided A, Strided B, StridedOut C, int splits,
           double* partials, cudaStream_t s, Launches& L);
void gen_start_basis(double* Z, int F, int k, uint64_t seed, cudaStream_t s, Launches& L);
// Q = qr(Z) by shifted CholeskyQR3, batch of 3, in place on Z (Z -> Q).
// Workspace of the orthonormalisation: Gram and factor [3][k][k], split-K
// partials, a copy of the input [3][F][k] and one flag per coordinate.
struct QrWork {
  double *G, *R, *partials, *save;
  uint32_t* bad;
  int splits;
  uint64_t seed;
};
// Z [3][F][k] <- its thin-QR factor Q.  `fill` ([3][F][k], e.g. the previous
// iterate, or null for seeded random vectors) completes the basis where Z is
// numerically rank deficient.
void cholqr3(double* Z, int F, int k, const QrWork& w, const double* fill, uint32_t* status,
             cudaStream_t s, Launches& L);
void oi_change(const double* Qold, const double* Qnew, int F, int k, double* work,
               double* change, cudaStream_t s, Launches& L);
// eigen-decomposition of H (3 x k x k): V (k x k, columns = eigenvectors,
// sorted descending), theta (k)
void jacobi_eig(const double* H, double* V, double* theta, int k, cudaStream_t s,
                Launches& L);
void sign_rule(double* U, int F, int k, cudaStream_t s, Launches& L);

// ---------------------------------------------------------------- tensor cores
// TMA descriptor (CUtensorMap, 128 bytes, 64-byte aligned storage at map_out)
// of a rows x K operand, K innermost, for tcgen05 tiles (128-byte swizzle).
bool tc_operand_map(void* map_out, const void* base, int elem_bytes, long long K, long long rows,
                    int batch, long long pitch, long long bpitch, int box_rows);
inline int tc_bn(int N) { return N <= 256 ? ((N + 15) / 16) * 16 : 256; }
size_t tc_smem_bytes(int BN);
// D = A B^T (FP32 accumulate) on tcgen05; kind 0 tf32, 1 bf16; returns splits used
// out_kind: 0 fp32, 1 fp32 rounded to tf32, 2 bf16, 3 fp64, 4 fp64 added to
// what out holds (one split only); element (m, n) of batch b / split z at
// out[b*sb + z*split_stride + m*s0 + n*s1]
int umma_tn(int kind, const void* mapA, const void* mapB, int M, int N, int K, int batch,
            int splits, void* out, int out_kind, long long s0, long long s1, long long sb,
            long long split_stride, uint32_t* status, cudaStream_t s, Launches& L);
void pack_operand_f64(const double* src, long long ssb, long long sr, long long sc, int batch,
                      long long rows, long long cols, long long dcols, long long dpitch,
                      long long dbp, int kind, void* dst, cudaStream_t s, Launches& L);
void pack_operand_f32(const float* src, long long ssb, long long sr, long long sc, int batch,
                      long long rows, long long cols, long long dcols, long long dpitch,
                      long long dbp, int kind, void* dst, cudaStream_t s, Launches& L);
void sum_splits(const float* part, int splits, long long stride, long long count, double* out,
                cudaStream_t s, Launches& L);

// ---------------------------------------------------------------- quantizer
struct Section {     // one coded section of the bitstream
  int bits;          // 0 = raw float64
  long long count;   // symbols
  long long offset;  // byte offset of the section in the stream
};
// lo/hi of row r of batch b: min/max over cols of A[b*s_batch + r*s_row + c*s_col],
// written to lo[b*out_sb + r] / hi[b*out_sb + r] (exact, order-free)
void minmax_rows_out(const double* A, long long rows, long long cols, long long s_row,
                     long long s_col, int batch, long long s_batch, double* lo, double* hi,
                     long long out_sb, cudaStream_t s, Launches& L);
// per coordinate c: min/max over all anchor values -> lo[c*out_sb], hi[c*out_sb]
void anchor_minmax_out(const double* X, const int32_t* anchors, int n_c, int F, double* lo,
                       double* hi, long long out_sb, cudaStream_t s, Launches& L);

struct EncodeLayout {
  int n, F, k, n_c, cb, db, ab, kind;
  long long total;
  long long anchors_off;
  long long coord_off[3];  // start of each coordinate block (its params)
  Section dict[3], coef[3], anch[3];
};
EncodeLayout make_layout(int n, int F, int k, int n_c, int cb, int db, int ab, int kind);
void write_header(uint8_t* out, const EncodeLayout& lay, const int32_t* anchors,
                  const double* qparams /*[3][4k+2]*/, cudaStream_t s, Launches& L);
void quant_pack_sections(uint8_t* out, const EncodeLayout& lay, const double* U,
                         const double* C, const double* X, const int32_t* anchors,
                         const double* qparams, cudaStream_t s, Launches& L);
void unpack_sections(const uint8_t* in, const EncodeLayout& lay, double* Udeq, double* Cdeq,
                     double* Ahat, int32_t* anchors, double* unused, uint32_t* status,
                     cudaStream_t s, Launches& L);

// ---------------------------------------------------------------- CG
struct CgState {
  double *rz, *rr, *bb, *pap, *alpha, *beta;  // [W]
  int32_t *done, *iters;                       // [W]
  double* partials;                            // [row_blocks * W * 2]
  int32_t* active;                             // [1] number of active columns
  int32_t* all_done;                           // [1]
};
struct CgGeom {
  int n, W, row_blocks, rows_per_block;
  // adjacency entries one row block can hold (rows_per_block x the largest
  // degree): the FP32 operator kernels stage their block's CSR slice in shared
  // memory when it is set; 0 reads the CSR from global memory
  int csr_cap;
};
CgGeom cg_geometry(int n, int W);
CgGeom cg_geometry_rows(int n, int W, int rows_per_block);
CgGeom cg_autotune(int n, int W, const int32_t* row_ptr, const int32_t* col_idx,
                   const int32_t* deg, const void* inv_d, const uint8_t* is_anchor, int kind,
                   void* P, void* T, void* Q, CgState& st, int single, cudaStream_t s,
                   Launches& L);
size_t cg_partials_elems(int n, int W);
// vectors X, R, P, T, Q are double (single = 0) or float (single = 1) [n][W]
// inv_d, inv_diag: double (single = 0) or float (single = 1) [n]
void cg_init(const CgGeom& g, const double* B, void* X, void* R, void* P,
             const void* inv_diag, CgState& st, int single, cudaStream_t s, Launches& L);
void cg_iteration(const CgGeom& g, const int32_t* row_ptr, const int32_t* col_idx,
                  const int32_t* deg, const void* inv_d, const uint8_t* is_anchor,
                  const void* inv_diag, int kind, void* X, void* R, void* P, void* T, void* Q,
                  double rtol, int max_iters, CgState& st, int single, cudaStream_t s,
                  Launches& L, cudaEvent_t* ev /* 7 events around the 6 kernels, or null */);
void widen(const float* X, long long count, double* out, cudaStream_t s, Launches& L);
// Iterative refinement of the CG solve (FP64 residuals, FP32 corrections):
// out[col] = ||B_col||^2; the FP64 residual R = B - M X of the unfrozen
// columns (T = L X as scratch), rr[col] = ||R_col||^2, frozen[col] set where
// rr <= rtol^2 bb or where the residual stalls below floor * ||X_col|| (prev:
// the last step's rr, reset to +inf by refine_reset), *active = number still
// open; X += D and the inner iteration counts added to total.
void refine_col_norms(const CgGeom& g, const double* B, double* partials, double* out,
                      cudaStream_t s, Launches& L);
void refine_reset(double* prev, int W, cudaStream_t s, Launches& L);
void refine_residual(const CgGeom& g, const int32_t* row_ptr, const int32_t* col_idx,
                     const int32_t* deg, const double* inv_d, const uint8_t* is_anchor, int kind,
                     const double* X, const double* B, double* T, double* R, int32_t* frozen,
                     double* partials, const double* bb, double rtol, double floor, double* prev,
                     double* rr, int32_t* active, cudaStream_t s, Launches& L);
void refine_update(const float* D, long long count, double* X, const int32_t* iters, int W,
                   int32_t* total, cudaStream_t s, Launches& L);
// Inner target of each column's correction: the relative reduction
// t = clamp(0.8 rtol ||B|| / ||R||, inner_rtol, 0.5) that brings the FP64
// residual below rtol ||B|| with a margin of 0.8, so no step solves further
// than the outer test needs; t2[col] = (t / inner_rtol)^2 (1 for frozen
// columns), and cg_bb[col] *= t2[col] when cg_bb is set (the CG's stop test
// rr <= inner_rtol^2 bb then stops at t)
void refine_targets(const double* rr, const double* bb, const int32_t* frozen, int W, double rtol,
                    double inner_rtol, double* t2, double* cg_bb, cudaStream_t s, Launches& L);
// CG start from the X already in place (warm start), T and Q as scratch
void cg_init_warm(const CgGeom& g, const int32_t* row_ptr, const int32_t* col_idx,
                  const int32_t* deg, const void* inv_d, const uint8_t* is_anchor, int kind,
                  const double* B, void* X, void* R, void* P, void* T, void* Q,
                  const void* inv_diag, CgState& st, int single, cudaStream_t s, Launches& L);
// FP32 CG with four columns per thread (W % 4 == 0), mc_cg4.cu
bool cg4_applies(int W, int single);
// One FP32 CG solve (column count a multiple of 4) of a batch whose solves
// advance together: grouped kernels cover every solve's (row block, column
// tile) items from a work table in one launch per phase.
struct CgSeq {
  CgGeom g;
  const int32_t *row_ptr, *col_idx, *deg;
  const float *inv_d, *inv_diag;
  const uint8_t* is_anchor;
  float *X, *R, *P, *T, *Q;
  double *partials, *rz, *rr, *bb, *alpha, *beta;
  int32_t *done, *iters, *active;
  int kind, max_iters;
  double rtol2;
};
constexpr int kGroupCols = 32;   // columns per grouped item (8 column lanes x 4)
// one grouped iteration: row items {solve, row block, column tile, 0}, column
// items {solve, column}; the counts are read from device memory, so a
// captured graph of iterations serves a shrinking table
void cg4_grouped_iteration(const CgSeq* seqs, const int4* items, const int* n_items,
                           const int2* cols, const int* n_cols, int grid_rows, int grid_cols,
                           size_t smem, cudaStream_t s, Launches& L);
void cgg_alpha(const CgSeq* seqs, const int2* cols, const int* n_cols, int grid, cudaStream_t s);
void cgg_beta(const CgSeq* seqs, const int2* cols, const int* n_cols, int grid, cudaStream_t s);
size_t cg4_grouped_smem(const CgGeom& g);
void cg4_init(const CgGeom& g, const double* B, float* X, float* R, float* P,
              const float* inv_diag, double* partials, cudaStream_t s);
void cg4_op(const CgGeom& g, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* deg,
            const float* inv_d, int kind, const uint8_t* is_anchor, const float* P, float* T,
            float* Q, const int32_t* done, double* partials, cudaStream_t s, cudaEvent_t* ev);
void cg4_update(const CgGeom& g, float* X, float* R, const float* P, const float* Q,
                const float* inv_diag, const double* alpha, const int32_t* done,
                double* partials, cudaStream_t s);
void cg4_dir(const CgGeom& g, const float* R, float* P, const float* inv_diag, const double* beta,
             const int32_t* done, cudaStream_t s);
void narrow(const double* X, long long count, float* out, cudaStream_t s, Launches& L);
constexpr int kCgKernels = 6;
extern const char* const kCgKernelNames[kCgKernels];
void scatter_anchor_rhs(double* B, const double* Ahat, const int32_t* anchors, int n_c, int F,
                        int W, int coord_cols, cudaStream_t s, Launches& L);
void factored_rhs(const double* Cdeq, int k, int n, int Wc, double* E, cudaStream_t s,
                  Launches& L);
void unit_anchor_columns(double* B, const int32_t* anchors, int n_c, int Wc, int col0,
                         cudaStream_t s, Launches& L);
void mark_anchors(const int32_t* anchors, int n_c, uint8_t* is_anchor, cudaStream_t s,
                  Launches& L);

}  // namespace mc
