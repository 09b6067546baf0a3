/*
 * mesh_codec.h - C ABI of the GB300 spatio-temporal dynamic-mesh codec.
 *
 * The codec follows "Fast Spatio-temporal Compression of Dynamic 3D Meshes"
 * (Arvanitis, Lalos, Moustakas).  Notation: n vertices with a fixed
 * triangle connectivity, F frames (the paper's k), rank k (the paper's k_l,
 * the number of retained rows of Eq. 10), n_c anchors (the paper's n_c,
 * index set N).
 *
 * Conventions for every entry point
 *   - Every pointer argument is owned by the caller and is only read or
 *     written during the call (and, for device pointers, by work the call
 *     enqueues on `stream`).  Nothing is retained after the call returns
 *     except inside the handle.
 *   - "device" pointers are CUDA global-memory addresses of the current
 *     device; "host" pointers are ordinary (pageable or pinned) host memory.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Device work is enqueued on it in order.
 *   - No entry point throws, aborts or traps; every failure is reported as a
 *     mesh_codec_status_t.  A handle is not thread-safe: use one handle per
 *     host thread and stream.
 *   - Sizes are in elements unless a name ends in `_bytes`.
 */
#ifndef MESH_CODEC_H
#define MESH_CODEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MESH_CODEC_API __attribute__((visibility("default")))
#else
#define MESH_CODEC_API
#endif

#define MESH_CODEC_ABI_VERSION 1
#define MESH_CODEC_MAX_RANK 64      /* k <= 64 */
#define MESH_CODEC_MAX_BITS 31      /* quantizer bits, 0 = raw binary64 */

typedef enum mesh_codec_status {
    MC_OK = 0,
    MC_E_INVALID_ARG = 1,        /* NULL pointer, size or parameter out of range */
    MC_E_BAD_MESH = 2,           /* triangle index out of range or repeated vertex */
    MC_E_ISOLATED_VERTEX = 3,    /* a vertex in no triangle: Eq. 3 divides by d_i = 0 */
    MC_E_OOM = 4,                /* device or pinned-host allocation failed */
    MC_E_CUDA = 5,               /* a CUDA runtime call failed */
    MC_E_NOT_CONVERGED = 6,      /* decoder solve hit its iteration cap; result written */
    MC_E_BITSTREAM_CORRUPT = 7,  /* header, sizes or anchor indices inconsistent */
    MC_E_BUFFER_TOO_SMALL = 8,   /* output capacity below the stream size; *written set */
    MC_E_NUMERICAL = 9,          /* an orthonormal basis could not be formed (non-finite
                                    input, or F above ~28,000 with rank-deficient data);
                                    numerically rank-deficient trajectories are completed,
                                    not rejected */
    MC_E_BAD_ANCHORS = 10,       /* caller-supplied anchors not strictly increasing in [0, n) */
    MC_E_NO_ANCHOR_IN_COMPONENT = 11, /* a connected component of the mesh holds no anchor:
                                    L 1 = 0 on every component (Eq. 3), so L^T L + P^T P
                                    of Eq. 12 is singular there; nothing is solved */
    MC_E_TIMEOUT = 12            /* a bounded wait inside a tensor-core kernel ran out
                                    (mesh_codec_set_wait_limit); the kernel drained its
                                    copies, freed its tensor memory and returned; the
                                    results of that call are not valid */
} mesh_codec_status_t;

/* Layout of the positions at the boundary (encode input, decode output,
 * the decoder's first iterate). */
typedef enum mesh_codec_layout {
    MC_LAYOUT_FRAMES = 0,        /* float64 [F][n][3]: frame-major, the sequence
                                    A = [M_1; ...; M_F] of Section II */
    MC_LAYOUT_VERTEX_MAJOR = 1   /* float64 [n][3][F]: one row of 3F values per vertex,
                                    coordinate c of frame f at column c*F + f (the
                                    codec's internal layout, so no transpose is run) */
} mesh_codec_layout_t;

/* Precision of the encoder's dense products and of the decoder's solve. */
typedef enum mesh_codec_precision {
    MC_PRECISION_FP64 = 0,       /* every step in binary64 */
    MC_PRECISION_TF32 = 1,       /* orthogonal-iteration sweeps, projection and
                                    back-projection on tcgen05 tensor cores with TF32
                                    operands and FP32 accumulation, then
                                    oi_refine_sweeps FP64 sweeps and the FP64
                                    Rayleigh-Ritz; QR, quantizer and solve stay FP64 */
    MC_PRECISION_BF16 = 2        /* the same with BF16 operands */
} mesh_codec_precision_t;

/* How the decoder forms the right-hand sides of Eq. 12. */
typedef enum mesh_codec_solve_mode {
    MC_SOLVE_FRAMES = 0,         /* one CG column per coordinate and frame (3F columns),
                                    the order of Eq. 11-12 */
    MC_SOLVE_FACTORED = 1,       /* 3k + n_c columns: M Y = L^T C'^T and M G = P^T, then
                                    X_c = Y_c U_c'^T + G a^_c (same solution, reassociated).
                                    The TF32 / BF16 modes split a^_c = (a^_c U_c') U_c'^T + E_c:
                                    Y_c also carries P^T a^_c U_c' and G multiplies only the
                                    anchors' residual E_c (still the same solution) */
    MC_SOLVE_AUTO = 2            /* FACTORED when 3k + n_c < 3F, or when the stream's
                                    anchors repeat the previous decode's (its anchor
                                    response G is then kept, and later decodes with
                                    those anchors solve 3k columns); else FRAMES.
                                    A decode given a first iterate keeps the first rule */
} mesh_codec_solve_mode_t;

typedef struct mesh_codec_params {
    int32_t n_vertices;          /* n >= 1 */
    int32_t n_triangles;         /* T >= 1 */
    int32_t n_frames;            /* F >= 1 (the paper's k) */
    int32_t rank;                /* k, 1 <= k <= min(F, MESH_CODEC_MAX_RANK) (the paper's k_l) */
    int32_t coeff_bits;          /* bits per coefficient symbol, 0..31 (0 = raw binary64); Eq. 10 */
    int32_t dict_bits;           /* bits per dictionary element; the paper assumes 16 */
    int32_t anchor_bits;         /* bits per anchor coordinate; the paper assumes 16 */
    int32_t n_anchors;           /* n_c, 0..n; 0 leaves Eq. 12 singular (rejected by decode) */
    int32_t laplacian_kind;      /* 0 = I - D^-1 C (Eq. 3, default), 1 = D - C (Eq. 1) */
    int32_t precision;           /* mesh_codec_precision_t */
    int32_t oi_sweeps;           /* orthogonal-iteration sweeps (maximum when oi_tol > 0) */
    int32_t cg_max_iters;        /* decoder CG iteration cap per column */
    double oi_tol;               /* stop when ||Q_new - Q Q^T Q_new||_F <= oi_tol; 0 = fixed count */
    double cg_rtol;              /* per-column stop: ||r|| <= cg_rtol * ||b|| */
    uint64_t seed;               /* anchors and the starting basis (splitmix64) */
    int32_t solve_mode;          /* mesh_codec_solve_mode_t */
    int32_t oi_refine_sweeps;    /* mixed precision: FP64 sweeps after the tensor-core ones */
    int32_t autotune;            /* 1: time candidate CG tile shapes on the first decode of each
                                    column count and keep the fastest (results then depend on
                                    the chosen shape at rounding level); 0: fixed shape */
    int32_t block_delta;         /* blocks variant (mesh_codec_encode_blocks): 1 = blocks
                                    2..n_b code their dictionary as the difference from
                                    the decoder's previous dictionary (Section IV, Fig. 6);
                                    0 = every block codes its own dictionary */
    int32_t block_delta_bits;    /* bits per dictionary difference, 0..31 (0 = raw binary64) */
    int32_t refine;              /* decoder solve: 0 = CG in the precision of the mode;
                                    r in 1..12 = iterative refinement: the residual of Eq. 12's
                                    normal equations in FP64, FP32 CG corrections solved to a
                                    relative 10^-r (a column whose residual needs less to meet
                                    cg_rtol stops at that, with a margin of 0.8), until every
                                    column's FP64 residual meets cg_rtol (FP64 accuracy from
                                    FP32 sweeps, any precision).
                                    In the TF32 / BF16 modes refine > 0 also keeps the
                                    projection (Eq. 9), the back-projection (Eq. 11) and the
                                    decoder's final products in FP64: the tensor cores then
                                    run only the orthogonal-iteration sweeps, which the FP64
                                    refinement sweeps and Rayleigh-Ritz correct */
    int32_t layout;              /* mesh_codec_layout_t of every positions argument; the
                                    blocks variant needs MC_LAYOUT_FRAMES */
    int32_t block_cg;            /* refined solve's inner solver (refine > 0 only):
                                    0 = one preconditioned CG per column; 1 = block CG
                                    (O'Leary): the columns in groups of 64 share one Krylov
                                    space, directions orthonormalised by CholeskyQR twice
                                    (FP32 vectors, FP64-summed Gram matrices, FP64 64 x 64
                                    algebra); the outer FP64 residual test is the same.
                                    The factored solves pad their columns to a multiple
                                    of 4 for it; a frames solve with 3F not a multiple of
                                    4 keeps the column CG */
} mesh_codec_params_t;

typedef struct mesh_codec_stats {
    int32_t oi_sweeps[3];        /* sweeps done per coordinate in the last encode */
    int32_t cg_iters_max;        /* over all CG columns of the last decode */
    int32_t cg_iters_min;
    int32_t cg_columns;          /* number of CG columns solved */
    int32_t cg_not_converged;    /* columns that hit cg_max_iters */
    int32_t cg_iterations_run;   /* CG iterations the last decode ran over all its columns
                                    (whole 32-iteration runs; the refined solve's inner
                                    iterations summed over its outer steps) */
    double oi_change[3];         /* last subspace change per coordinate (0 when not measured) */
    double cg_iters_mean;
    double cg_rel_residual_max;  /* max over columns of ||r|| / ||b|| (recursive residual) */
    uint64_t launches_create;    /* kernels launched by create / last encode / last decode */
    uint64_t launches_encode;
    uint64_t launches_decode;
    uint64_t workspace_bytes;    /* device memory held by the handle */
} mesh_codec_stats_t;

typedef struct mesh_codec mesh_codec_t;   /* opaque handle */

/* Human-readable name of a status code (static storage, never NULL). */
MESH_CODEC_API const char* mesh_codec_status_string(mesh_codec_status_t s);

/* Fills *p with defaults: 12/16/16 bits, random-walk Laplacian, FP64,
 * 30 sweeps, cg_rtol 1e-14, cg_max_iters 50000, seed 0, solve_mode FRAMES.
 * Sizes (n, T, F, k, n_c) are zeroed and must be set by the caller. */
MESH_CODEC_API void mesh_codec_default_params(mesh_codec_params_t* p);

/* Creates a codec for one fixed connectivity (the paper's L is built once
 * from it and is the same for all frames, Section III).
 *   triangles: int32 [T][3], 0-based vertex indices, host or device
 *              (`triangles_on_device`).
 *   anchors:   NULL to draw n_c anchors from `seed` (the n_c vertices with the
 *              smallest splitmix64 keys), or int32 [n_c] strictly increasing
 *              indices in [0, n), host or device (`anchors_on_device`).
 * Builds the CSR adjacency, degrees, the anchor set, the starting basis and
 * allocates the device workspace for (n, F, k).  Labels the connected
 * components of the mesh; with n_c > 0 every component must hold an anchor
 * (Eq. 12 is singular otherwise), with n_c = 0 the handle can only encode.
 * Synchronises `stream`.
 * Errors: MC_E_INVALID_ARG, MC_E_BAD_MESH, MC_E_ISOLATED_VERTEX,
 * MC_E_BAD_ANCHORS, MC_E_NO_ANCHOR_IN_COMPONENT, MC_E_OOM, MC_E_CUDA,
 * MC_E_NUMERICAL; *out is NULL then. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_create(const mesh_codec_params_t* params,
                                      const int32_t* triangles, int triangles_on_device,
                                      const int32_t* anchors, int anchors_on_device,
                                      void* stream, mesh_codec_t** out);

/* Anchors spread evenly over a pose (Section III-B asks for n_c uniformly
 * distributed anchor vertices; mesh_codec_create draws them at random when
 * given none): greedy farthest-point selection in Euclidean distance.  From
 * vertex `start`, n_c - 1 times the vertex farthest from its nearest chosen
 * vertex joins the set (squared distances formed as (dx*dx + dy*dy) + dz*dz,
 * every operation rounded separately; equal distances: the lower index).
 *   xyz:     device float64 [n][3], e.g. the first frame of the sequence.
 *   anchors: device int32 [n_c], written in ascending order, ready for
 *            mesh_codec_create.
 * Needs 1 <= n_c <= n and 0 <= start < n.  Allocates its scratch (8n + 4n_c
 * bytes and about 10 KB) on `stream` and frees it there; one kernel launch
 * per anchor.  Errors: MC_E_INVALID_ARG, MC_E_OOM, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_farthest_anchors(int n, int n_c, const double* xyz,
                                                               int start, int32_t* anchors,
                                                               void* stream);

/* Exact size in bytes of every bitstream this handle produces. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_encoded_size(const mesh_codec_t* h, size_t* bytes);

/* Encoder (Section III, Eq. 7-10).
 *   positions: device float64 [F][n][3] (frame-major, the sequence
 *              A = [M_1; ...; M_F] of Section II), or [n][3][F] with
 *              params.layout = MC_LAYOUT_VERTEX_MAJOR.
 *   bitstream: device bytes, `capacity` of them, 8-byte aligned; receives
 *              the stream: a 64-byte header ("DMC1", version 1, n, F, k,
 *              n_c, the three bit counts, the Laplacian kind, the total
 *              size), the anchor indices, then per coordinate the quantizer
 *              ranges (f64 lo/hi per dictionary column, per coefficient row,
 *              and for the anchors) and three symbol sections (dictionary in
 *              column-major order, coefficients row-major, anchors
 *              anchor-major), each packed as bit planes of 32-symbol groups
 *              (word g*b + j holds bit j of symbols 32g..32g+31) and padded
 *              to 8 bytes; raw binary64 values when a bit count is 0.
 *   written:   host; set to the stream size, also on MC_E_BUFFER_TOO_SMALL
 *              (nothing is enqueued then).
 * Synchronises `stream` once at the end to read the device status word.
 * Errors: MC_E_INVALID_ARG, MC_E_BUFFER_TOO_SMALL, MC_E_NUMERICAL,
 * MC_E_TIMEOUT, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_encode(mesh_codec_t* h, const double* positions,
                                      uint8_t* bitstream, size_t capacity, size_t* written,
                                      void* stream);

/* Decoder (Eq. 11-12, parallel anchored reconstruction over all frames).
 *   bitstream:     device bytes, `bytes` of them, produced by a handle with
 *                  the same parameters and connectivity.
 *   positions_out: device float64 [F][n][3] (or [n][3][F] with
 *                  MC_LAYOUT_VERTEX_MAJOR).
 * Reads the 64-byte header back to the host (one synchronisation), checks
 * that the stream's anchors hold one vertex of every connected component
 * (a second one; MC_E_NO_ANCHOR_IN_COMPONENT before any solve work
 * otherwise) and reads the status word at the end (a third one).
 * MC_E_NOT_CONVERGED still writes the best iterate.
 * Errors: MC_E_INVALID_ARG, MC_E_BITSTREAM_CORRUPT,
 * MC_E_NO_ANCHOR_IN_COMPONENT, MC_E_NOT_CONVERGED, MC_E_TIMEOUT, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_decode(mesh_codec_t* h, const uint8_t* bitstream, size_t bytes,
                                      double* positions_out, void* stream);

/* Decoder with a warm start: `x0` (device float64 [F][n][3], or NULL for the
 * cold start X0 = 0) is the first iterate of the CG solve of Eq. 12, e.g. the
 * previous segment's reconstruction or a learned prediction of it.  The
 * result is the same least-squares solution; only the iteration count
 * changes.  Needs solve_mode FRAMES (the factored solve has no X iterate).
 * Errors: as mesh_codec_decode, MC_E_INVALID_ARG for a misaligned x0 or a
 * factored handle. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_decode_ex(mesh_codec_t* h, const uint8_t* bitstream,
                                                        size_t bytes, const double* x0,
                                                        double* positions_out, void* stream);

/* The first stage of the decoder alone: unpack and dequantize the stream
 * (Eq. 10) and, when `delta_out` is not NULL, back-project the delta
 * coordinates (Eq. 11) into it (device float64 [n][3F], vertex-major,
 * column c*F + f); when `anchors_out` is not NULL, copy the dequantized
 * anchor positions there (device float64 [3][n_c][F]).  No solve.  Lets a
 * caller build a warm start for mesh_codec_decode_ex from what the stream
 * carries.  Synchronises `stream`.  Errors: as mesh_codec_decode. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_decode_stage(mesh_codec_t* h, const uint8_t* bitstream,
                                                           size_t bytes, double* delta_out,
                                                           double* anchors_out, void* stream);

/* Start basis of the orthogonal iterations (Algorithm 1).  `q0`: device
 * float64 [3][F][k], made orthonormal (CholeskyQR3; columns dependent on
 * earlier ones are replaced by seeded random directions) and used by every
 * following encode, e.g. the previous block's dictionary U[i-1] as
 * Algorithm 1 does for blocks 2..n_b; NULL restores the seeded random start.
 * Synchronises `stream`.  Errors: MC_E_INVALID_ARG, MC_E_NUMERICAL
 * (non-finite q0), MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_set_start_basis(mesh_codec_t* h, const double* q0,
                                                              void* stream);

/* Blocks variant (Section III-A, Algorithm 1).  A sequence of
 * n_blocks * F frames (F = the handle's n_frames, the paper's k_f) is coded
 * as n_blocks consecutive blocks with the handle's connectivity, anchors and
 * parameters:
 *   block 1: U[1] from the eigendecomposition of R[1] = A A^T (Algorithm 1's
 *            SVD; F <= 64; for F > 64 the seeded one-block iterations);
 *   block i >= 2: oi_sweeps sweeps Q <- QR(R[i] Q) from Q = U[i-1]
 *            (Algorithm 1), then Rayleigh-Ritz and signs as for one block;
 *   with params.block_delta, blocks i >= 2 code U[i] - U^[i-1] (U^ the
 *            dequantized dictionary the decoder holds) in block_delta_bits.
 * Container: 64-byte header (magic "DMCB", u32 version 1, u32 n_blocks,
 * u32 flags (bit 0: differences), u32 delta bits, u64 first block bytes,
 * u64 other block bytes, u64 total bytes, zero padding), then the block
 * streams in order, each a version-1 stream of mesh_codec_encode.
 * mesh_codec_blocks_size gives the container size for n_blocks. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_blocks_size(const mesh_codec_t* h, int n_blocks,
                                                          size_t* bytes);

/* Bits per vertex and frame of the streams a handle with parameters *p
 * writes, for n_blocks blocks of p->n_frames frames (1: a plain stream), as
 * the terms of Eq. 13 for what the stream holds (k of the F dictionary
 * columns per block):
 *   out[0] q   = coeff_bits * k / F
 *   out[1] q_a = anchor_bits * n_c / n
 *   out[2] q_d = dictionary bits * k / n, averaged over the blocks (block 1
 *                dict_bits; blocks 2..n_b block_delta_bits when block_delta)
 *   out[3] q_s = q + q_a + q_d
 *   out[4] the stream's own rate: its bytes * 8 / (n * F * n_blocks), with
 *          headers, anchor indices, quantizer ranges and padding
 * (a bit count of 0 means raw binary64: 64 bits).  Host arithmetic only: no
 * device is used.  Errors: MC_E_INVALID_ARG. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_rates(const mesh_codec_params_t* p, int n_blocks,
                                                    double* out);

/* positions: device float64 [n_blocks * F][n][3]; out: device, 8-byte
 * aligned, `capacity` bytes; *written = the container size (also on
 * MC_E_BUFFER_TOO_SMALL).  Leaves the handle's start basis unchanged.
 * Synchronises `stream` at the end.  Errors: as mesh_codec_encode. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_encode_blocks(mesh_codec_t* h,
                                                            const double* positions,
                                                            int n_blocks, uint8_t* out,
                                                            size_t capacity, size_t* written,
                                                            void* stream);

/* Decodes a container of mesh_codec_encode_blocks into positions_out
 * (device float64 [n_blocks * F][n][3], n_blocks from the container).  In
 * the frames solve mode each block's CG starts from the previous block's
 * last decoded frame (same solution, fewer iterations).  Errors: as
 * mesh_codec_decode; MC_E_BITSTREAM_CORRUPT for a container whose sizes or
 * flags do not match the handle. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_decode_blocks(mesh_codec_t* h, const uint8_t* in,
                                                            size_t bytes, double* positions_out,
                                                            void* stream);

/* Same as encode / decode with HOST buffers: the call copies the input to
 * the device, runs the codec and copies the result back before returning.
 * Host memory may be pageable; pinned memory copies faster. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_encode_host(mesh_codec_t* h, const double* positions_host,
                                           uint8_t* bitstream_host, size_t capacity,
                                           size_t* written, void* stream);
MESH_CODEC_API mesh_codec_status_t mesh_codec_decode_host(mesh_codec_t* h, const uint8_t* bitstream_host,
                                           size_t bytes, double* positions_out_host,
                                           void* stream);

/* Batches of independent sequences (each with its own handle, connectivity
 * and sizes).  The work of handle i runs on a stream of its own, forked from
 * and joined back to `stream` with events, so that sequences of uneven size
 * overlap on the GPU; the decoders' CG solves advance in lockstep runs of 32
 * iterations, each replayed from the handle's CUDA graph.  Arrays have
 * `count` entries; a handle may appear once.  `written[i]` / `statuses[i]`
 * (statuses may be NULL) receive the per-sequence results; the return value
 * is the first non-OK status.  Synchronises every handle's stream before
 * returning. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_encode_batch(mesh_codec_t* const* handles,
                                                           int count,
                                                           const double* const* positions,
                                                           uint8_t* const* bitstreams,
                                                           const size_t* capacities,
                                                           size_t* written,
                                                           mesh_codec_status_t* statuses,
                                                           void* stream);
MESH_CODEC_API mesh_codec_status_t mesh_codec_decode_batch(mesh_codec_t* const* handles,
                                                           int count,
                                                           const uint8_t* const* bitstreams,
                                                           const size_t* bytes,
                                                           double* const* positions_out,
                                                           mesh_codec_status_t* statuses,
                                                           void* stream);
/* mesh_codec_decode_batch with flags.  MC_BATCH_GROUPED: the FP32 solves
 * whose column count is a multiple of 4 (the mixed modes' factored solves,
 * frames solves with F % 4 == 0) advance as grouped batches - the solves are
 * dealt, largest first, over up to four batches on streams of their own, and
 * every phase of a batch's iteration is one launch over a work table of
 * (sequence, row block, column tile) and (sequence, column) items, one CTA
 * per item, 32 iterations replayed from one CUDA graph, finished sequences
 * leaving the table between runs; the other solves run on their own streams
 * alongside.  A grouped sequence's result equals its result alone (same
 * arithmetic, tile shape and reduction order).  0 is mesh_codec_decode_batch.
 * Errors: as mesh_codec_decode_batch; MC_E_INVALID_ARG for unknown flags. */
#define MC_BATCH_GROUPED 1
MESH_CODEC_API mesh_codec_status_t mesh_codec_decode_batch_ex(mesh_codec_t* const* handles,
                                                              int count,
                                                              const uint8_t* const* bitstreams,
                                                              const size_t* bytes,
                                                              double* const* positions_out,
                                                              mesh_codec_status_t* statuses,
                                                              int flags, void* stream);

/* Statistics of the last create / encode / decode (synchronises the handle's
 * last stream). */
MESH_CODEC_API mesh_codec_status_t mesh_codec_get_stats(const mesh_codec_t* h, mesh_codec_stats_t* st);

/* Internal buffers, for inspection and testing.  Copies `count` elements of
 * buffer `which` into the device buffer `dst` (enqueued on `stream`).
 * `count` must equal the buffer's size, which mesh_codec_buffer_size reports.
 *   MC_BUF_ROW_PTR   int32 [n+1]      CSR row offsets of the adjacency (no diagonal)
 *   MC_BUF_COL_IDX   int32 [nnz]      column indices, ascending within each row
 *   MC_BUF_DEGREE    int32 [n]        d_i = |Psi_i|
 *   MC_BUF_ANCHORS   int32 [n_c]      anchor indices, ascending
 *   MC_BUF_DELTA     float64 [n][3F]  delta coordinates of the last encode, vertex-major
 *                                     (column c*F + f = coordinate c, frame f)
 *   MC_BUF_BASIS     float64 [3][F][k] the dictionaries U_c of the last encode
 *   MC_BUF_RITZ      float64 [3][k]   Ritz values (descending) of the last encode
 *   MC_BUF_COEFF     float64 [3][k][n] the projections C_c = U_c^T delta_c^T (Eq. 9)
 *   MC_BUF_START     float64 [3][F][k] the starting bases Q0_c
 *   MC_BUF_DELTA_REC float64 [n][3F]  decoded delta coordinates of the last decode (FRAMES
 *                                     mode; the FACTORED decode leaves X there instead)
 *   MC_BUF_CG_ITERS  int32 [columns]  CG iterations per column of the last decode */
typedef enum mesh_codec_buffer {
    MC_BUF_ROW_PTR = 0, MC_BUF_COL_IDX = 1, MC_BUF_DEGREE = 2, MC_BUF_ANCHORS = 3,
    MC_BUF_DELTA = 4, MC_BUF_BASIS = 5, MC_BUF_RITZ = 6, MC_BUF_COEFF = 7,
    MC_BUF_START = 8, MC_BUF_DELTA_REC = 9, MC_BUF_CG_ITERS = 10
} mesh_codec_buffer_t;

MESH_CODEC_API mesh_codec_status_t mesh_codec_buffer_size(const mesh_codec_t* h, int which,
                                           size_t* count, size_t* elem_bytes);
MESH_CODEC_API mesh_codec_status_t mesh_codec_copy_buffer(const mesh_codec_t* h, int which,
                                           void* dst, size_t count, void* stream);

/* Kernel timing.  With `every` > 0, each decode records CUDA events on its
 * stream around the kernels of sampled CG iterations and adds their
 * durations to per-kernel totals; 0 turns it off.  A full run of 32
 * iterations whose first iteration's index is a multiple of `every` samples
 * its last iteration (the 31 before it replay from a CUDA graph, as without
 * timing, and the timed launches queue behind them); shorter runs sample
 * every `every`-th iteration.  The refined solve's inner runs do the same
 * with direct launches.  The last entry of the profile, "cg_iteration",
 * holds the whole iterations that ran between one event pair with no
 * events inside (the 31-iteration graph replays, the first iterations of
 * each refined run): launches_timed counts those iterations and total_ms
 * their time, i.e. the iteration time without per-kernel events.
 * Sampling leaves the results unchanged.  Either call resets the totals.
 * mesh_codec_get_profile synchronises the handle's last stream. */
#define MESH_CODEC_PROF_KERNELS 8
typedef struct mesh_codec_profile {
    int32_t n_kernels;
    int32_t reserved;
    char name[MESH_CODEC_PROF_KERNELS][32];
    int64_t launches_timed[MESH_CODEC_PROF_KERNELS];
    double total_ms[MESH_CODEC_PROF_KERNELS];
} mesh_codec_profile_t;
MESH_CODEC_API mesh_codec_status_t mesh_codec_set_profiling(mesh_codec_t* h, int every);
MESH_CODEC_API mesh_codec_status_t mesh_codec_get_profile(const mesh_codec_t* h,
                                                          mesh_codec_profile_t* out);

/* Test entry point for the tensor-core GEMM behind the mixed-precision modes:
 * C (M x N, float64) = A (M x K) * B^T with A, B float32 device row-major
 * [M][K] and [N][K], operands rounded to TF32 (kind 0) or BF16 (kind 1),
 * products accumulated in FP32 on tcgen05 tensor cores per K split, splits
 * summed in FP64.  Allocates and frees its own temporaries; synchronises
 * `stream`.  Errors: MC_E_INVALID_ARG, MC_E_OOM, MC_E_TIMEOUT, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_selftest_gemm(int kind, int M, int N, int K,
                                                            int splits, const float* A,
                                                            const float* B, double* C,
                                                            void* stream);

/* Limit, in nanoseconds of the GPU's global timer, on every wait of the
 * tensor-core kernels (a copy landing in shared memory, the products that
 * read a stage completing); 0 restores the default of 2 s.  Process-wide;
 * read when a kernel is launched.  A wait that runs out makes its block
 * record a timeout, wait (again bounded) for its copies and products in
 * flight, free its tensor memory and return; the call then reports
 * MC_E_TIMEOUT and the next call proceeds normally.  A limit of a few
 * microseconds makes the waits of a long product run out on purpose, which
 * is how the timeout path is tested.  Errors: none (always MC_OK). */
MESH_CODEC_API mesh_codec_status_t mesh_codec_set_wait_limit(unsigned long long ns);

/* Adjacency build that allocates nothing.  The paper has no counterpart:
 * this is a service for callers that cannot call cudaMalloc where they need
 * a mesh's adjacency, such as real-time hosts that make every allocation
 * before their processing loop starts (an allocation can block for
 * milliseconds and synchronise the device), or plug-ins whose device memory
 * belongs to another framework's caching allocator (a cudaMalloc of their
 * own can fail or fragment the pool that framework manages).
 *
 * Builds the same CSR adjacency as mesh_codec_create (MC_BUF_ROW_PTR,
 * MC_BUF_COL_IDX, MC_BUF_DEGREE): every row sorted ascending, duplicates
 * and the diagonal removed.
 *   triangles:        device int32 [n_triangles][3], 0-based.
 *   row_ptr:          device int32 [n_vertices + 1], written.
 *   col_idx:          device int32 [col_idx_capacity]; nnz entries written.
 *   deg:              device int32 [n_vertices], written.
 *   nnz_out:          host; the number of adjacency entries (row_ptr[n]),
 *                     also set on MC_E_BUFFER_TOO_SMALL.
 * Limits: n_vertices <= MESH_CODEC_STATIC_MAX_VERTICES and n_triangles <=
 * MESH_CODEC_STATIC_MAX_TRIANGLES; larger sizes return MC_E_INVALID_ARG
 * before any work is enqueued.
 * Memory: the call allocates no device or host memory (no cudaMalloc,
 * cudaFree or allocating library call).  Its scratch is a static device
 * array of 7,865,344 bytes (7.5 MiB) inside the library, which every GPU that loads the
 * library holds until the process exits.  All calls share that array and it
 * keeps the last call's contents; the call clears what must start at zero.
 * Calls whose GPU work overlaps (other host threads, or streams not ordered
 * with this one) race on it and must be serialised by the caller.
 * The first call on each device (and again in each new CUDA context of that
 * device, e.g. after cudaDeviceReset) looks up the array's device address
 * with that device current; make that first call before any stream capture.
 * Synchronises `stream` once (to read nnz and the error word); the
 * compaction of col_idx is enqueued after that and is complete in stream
 * order.  Errors: MC_E_INVALID_ARG, MC_E_BAD_MESH, MC_E_ISOLATED_VERTEX,
 * MC_E_BUFFER_TOO_SMALL, MC_E_CUDA. */
#define MESH_CODEC_STATIC_MAX_VERTICES (1 << 17)
#define MESH_CODEC_STATIC_MAX_TRIANGLES (1 << 18)
MESH_CODEC_API mesh_codec_status_t mesh_codec_adjacency_static(const int32_t* triangles,
                                                               int n_triangles, int n_vertices,
                                                               int32_t* row_ptr, int32_t* col_idx,
                                                               size_t col_idx_capacity,
                                                               int32_t* deg, int32_t* nnz_out,
                                                               void* stream);

/* Frees the handle and its workspace (synchronises the device first).
 * NULL is accepted. */
MESH_CODEC_API void mesh_codec_destroy(mesh_codec_t* h);

/* ------------------------------------------------------------------------
 * Learned warm start for the decoder.  The paper has no counterpart: its
 * decoder solves Eq. 12 from scratch.  A small perceptron predicts each
 * segment's positions from the previous segment's reconstruction and the
 * current segment's anchors and delta coordinates; the prediction is passed
 * to mesh_codec_decode_ex as the CG's first iterate, so it changes only the
 * iteration count, never the solution.
 *
 * Network: n_in -> n_hidden -> n_hidden -> n_out on standardised inputs
 * (mesh_codec_mlp_fit_normalizer), ReLU after the two hidden layers, none
 * after the output.  Parameters are one flat float32 array
 * [W1 (n_hidden x n_in, row-major), b1, W2 (n_hidden x n_hidden), b2,
 *  W3 (n_out x n_hidden), b3]; every product uses a bfloat16 copy of the
 * weights (round to nearest even) with float32 accumulation; biases stay
 * float32.  Training minimises the mean squared error over all outputs with
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the float32 master copy.
 * Samples are rows: X [N][n_in], targets and outputs [N][n_out], float32,
 * device memory, row-major.  One handle is not safe for concurrent calls.
 * ---------------------------------------------------------------------- */
typedef struct mesh_codec_mlp mesh_codec_mlp_t;

/* Allocates a network with He-uniform weights drawn from splitmix64(seed)
 * (output layer scaled by 0.1) and zero biases; synchronises the device.
 * Sizes 1..4096.  Errors: MC_E_INVALID_ARG, MC_E_OOM, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_mlp_create(int n_in, int n_hidden, int n_out,
                                                         uint64_t seed, mesh_codec_mlp_t** out);

/* Number of float32 parameters (0 for NULL). */
MESH_CODEC_API size_t mesh_codec_mlp_param_count(const mesh_codec_mlp_t* m);

/* Copies parameter_count floats to device `dst`: which = 0 the float32
 * master parameters, 1 the bfloat16 copy widened to float32, 2 the gradient
 * of the last mesh_codec_mlp_train_step.  Errors: MC_E_INVALID_ARG, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_mlp_get_params(const mesh_codec_mlp_t* m, int which,
                                                             float* dst, void* stream);

/* Replaces the master parameters (device float32, parameter_count values),
 * refreshes the bfloat16 copy and resets Adam's moments and step count.
 * Errors: MC_E_INVALID_ARG, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_mlp_set_params(mesh_codec_mlp_t* m, const float* src,
                                                             void* stream);

/* Y = network(X) for N rows, enqueued on `stream`, in chunks of at most
 * 4,194,304 rows.  Grows the handle's activation buffers to one chunk on
 * first use of a larger N (cudaMalloc).
 * Errors: MC_E_INVALID_ARG, MC_E_OOM, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_mlp_forward(mesh_codec_mlp_t* m, const float* X,
                                                          long long N, float* Y, void* stream);

/* Inference: the network of mesh_codec_mlp_forward with its hidden-to-hidden
 * product (n_hidden^2 of its multiply-adds per row) on the tcgen05 tensor
 * cores as a TF32 GEMM: the bfloat16 weights enter exactly, the float32
 * activations are rounded to TF32 (10-bit mantissa) by the MMA, the products
 * accumulate in float32.  Outputs agree with mesh_codec_mlp_forward to
 * about 1e-3 of their scale.  For predictions over many rows (the warm
 * start's first iterate); training and the gradient checks use the
 * float32-product forward.  It uses the bfloat16 weights whatever the check
 * mode (mesh_codec_mlp_set_check_mode).  Synchronises `stream` to read the tensor-core
 * status; when n_hidden is not a multiple of 4 (no TMA description) it runs
 * mesh_codec_mlp_forward.  Errors: MC_E_INVALID_ARG, MC_E_OOM, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_mlp_infer(mesh_codec_mlp_t* m, const float* X,
                                                        long long N, float* Y, void* stream);

/* Forward pass, loss mean((Y - T)^2) and its gradient for N rows; with
 * update != 0 one Adam step of learning rate lr.  `loss` (host, may be
 * NULL) receives the loss, which synchronises `stream`.
 * Errors: MC_E_INVALID_ARG, MC_E_OOM, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_mlp_train_step(mesh_codec_mlp_t* m, const float* X,
                                                             const float* T, long long N, float lr,
                                                             int update, double* loss,
                                                             void* stream);

/* Input standardisation: the network reads x' = (x - mu) * inv_sigma per
 * feature (float32), identity (mu 0, inv_sigma 1) until fitted.  Fitting
 * sets mu to the column means of X [N][n_in] and inv_sigma to 1 / the
 * population standard deviation (sums in float64; a column with standard
 * deviation <= 1e-12 * max(1, |mean|) keeps inv_sigma = 1).
 * Errors: MC_E_INVALID_ARG, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_mlp_fit_normalizer(mesh_codec_mlp_t* m,
                                                                 const float* X, long long N,
                                                                 void* stream);
/* Copies mu and inv_sigma (n_in float32 each) to device memory. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_mlp_get_normalizer(const mesh_codec_mlp_t* m,
                                                                 float* mu, float* inv_sigma,
                                                                 void* stream);

/* Check mode: fp32_weights = 1 makes every product read the float32 master
 * weights instead of the bfloat16 copy (for gradient checks against a
 * float64 reference); 0 (the default) restores bfloat16.
 * Errors: MC_E_INVALID_ARG. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_mlp_set_check_mode(mesh_codec_mlp_t* m,
                                                                 int fp32_weights);

/* Frees the network (synchronises the device first).  NULL is accepted. */
MESH_CODEC_API void mesh_codec_mlp_destroy(mesh_codec_mlp_t* m);

/* For each vertex v of a rest pose `rest` (device float64 [n][3]) the
 * indices into `anchors` (device int32 [n_c]) of its MESH_CODEC_WARM_ANCHORS
 * nearest anchors in Euclidean distance, nearest first (equal distances:
 * the lower index first; with fewer anchors the last one repeats), written
 * to nearest[v][j] (int32), and those distances to dist[v][j] (float32).
 * Errors: MC_E_INVALID_ARG, MC_E_CUDA. */
#define MESH_CODEC_WARM_ANCHORS 3
#define MESH_CODEC_WARM_FEATURES 16
MESH_CODEC_API mesh_codec_status_t mesh_codec_nearest_anchor(int n, int n_c, const double* rest,
                                                             const int32_t* anchors,
                                                             int32_t* nearest, float* dist,
                                                             void* stream);

/* Warm-start features of segment s from what its stream carries and the
 * decoded segment s-1: MESH_CODEC_WARM_FEATURES float32 per sample, sample
 * index e = f*n + v, for the nearest anchors a_j = nearest[v][j]:
 *   [4j .. 4j+2] a_cur(a_j, f) - x_last(anchors[a_j])   (j = 0, 1, 2)
 *   [4j + 3]     dist[v][j]
 *   [12 .. 14]   (delta_cur(v, f) - delta_prev(v, F-1)) * dscale
 *   [15]         (f + 1) / F
 * x_last: the last decoded frame of segment s-1, device float64 [n][3].
 * a_cur: the dequantized anchor positions of segment s, [3][n_c][F];
 * delta_cur, delta_prev: the back-projected delta coordinates of segments s
 * and s-1, vertex-major [n][3F] (column c*F + f), as mesh_codec_decode_stage
 * returns them.  With x_cur ([F][n][3]) != NULL also writes the regression
 * target target[e][c] = x_cur(v, f) - x_last(v) (float32 [n*F][3]).
 * Each difference is formed in float64 and rounded once to float32.
 * Errors: MC_E_INVALID_ARG, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_warm_features(
    int n, int F, int n_c, const double* x_last, const double* a_cur, const int32_t* anchors,
    const int32_t* nearest, const float* dist, const double* delta_cur, const double* delta_prev,
    float dscale, const double* x_cur, float* features, float* target, void* stream);

/* Decoder start from a prediction: x0(f, v, c) = x_last(v, c) + pred[f*n + v][c]
 * (float64 [F][n][3]); pred (float32 [n*F][3]) may be NULL for the plain
 * previous-frame start.  Errors: MC_E_INVALID_ARG, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_warm_compose(int n, int F, const double* x_last,
                                                           const float* pred, double* x0,
                                                           void* stream);

/* Training minibatch: out[i][:] = X[r_i][:] for i < count, rows of `width`
 * float32, r_i = splitmix64(seed) output i modulo N.  Equal seeds draw equal
 * rows, so features and targets are sampled by two calls with one seed.
 * Errors: MC_E_INVALID_ARG, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_sample_rows(const float* X, int width, long long N,
                                                          uint64_t seed, long long count,
                                                          float* out, void* stream);

/* Basis head of the warm start (the encoder's Algorithm 1 start).  Row
 * r = c*F + f of the previous segment's dictionary U_prev (device float64
 * [3][F][k], as MC_BUF_BASIS holds it) gives the features
 * [U_prev(c, f, 0..k-1), (f + 1) / F] (float32 [3F][k+1]); with U_cur !=
 * NULL also the target U_cur - U_prev (float32 [3F][k]).
 * Errors: MC_E_INVALID_ARG, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_basis_features(int F, int k, const double* U_prev,
                                                             const double* U_cur, float* features,
                                                             float* target, void* stream);

/* q0 = U_prev + pred (float64 [3][F][k]; pred float32 [3F][k] or NULL), to
 * pass to mesh_codec_set_start_basis.  Errors: MC_E_INVALID_ARG, MC_E_CUDA. */
MESH_CODEC_API mesh_codec_status_t mesh_codec_basis_compose(int F, int k, const double* U_prev,
                                                            const float* pred, double* q0,
                                                            void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MESH_CODEC_H */
