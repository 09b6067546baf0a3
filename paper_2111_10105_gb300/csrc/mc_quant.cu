// Quantization and bit-plane packing of the bitstream (Eq. 10 and the
// dictionary / anchor coding of Section IV), and the decoder's inverse.
//
// Q(.) is a uniform scalar quantizer per group (coefficient row, dictionary
// column, all anchor values of one coordinate): range = hi - lo,
// scale = (2^b - 1) / range, s = floor((x - lo) * scale + 0.5) clamped to
// [0, 2^b - 1], every operation separately rounded (no fused multiply-add),
// so the symbol is decided in binary64 exactly as written.  Reconstruction
// x^ = lo + s * (range / (2^b - 1)).
//
// Packing: a warp codes a group of 32 consecutive symbols; bit plane j of
// the group is one __ballot_sync, stored as word g*b + j (lane l = symbol
// 32g + l).  Words are little-endian uint32; a section is padded to 8 bytes.
#include <algorithm>
#include <math.h>

#include "mc_internal.cuh"

namespace mc {

static long long pad8(long long b) { return (b + 7) / 8 * 8; }
static long long packed_words(long long count, int bits) { return ((count + 31) / 32) * bits; }
static long long section_bytes(long long count, int bits) {
  return bits == 0 ? count * 8 : pad8(packed_words(count, bits) * 4);
}

EncodeLayout make_layout(int n, int F, int k, int n_c, int cb, int db, int ab, int kind) {
  EncodeLayout L{};
  L.n = n; L.F = F; L.k = k; L.n_c = n_c; L.cb = cb; L.db = db; L.ab = ab; L.kind = kind;
  long long off = 64;
  L.anchors_off = off;
  off += pad8(4LL * n_c);
  for (int c = 0; c < 3; ++c) {
    L.coord_off[c] = off;
    off += 8LL * (4LL * k + 2);
    L.dict[c] = Section{db, (long long)F * k, off};
    off += section_bytes((long long)F * k, db);
    L.coef[c] = Section{cb, (long long)k * n, off};
    off += section_bytes((long long)k * n, cb);
    L.anch[c] = Section{ab, (long long)n_c * F, off};
    off += section_bytes((long long)n_c * F, ab);
  }
  L.total = off;
  return L;
}

// ------------------------------------------------------------ min / max
__device__ __forceinline__ void block_minmax(double& lo, double& hi) {
  __shared__ double slo[32], shi[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
  }
  if (lane == 0) { slo[warp] = lo; shi[warp] = hi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { lo = fmin(lo, slo[w]); hi = fmax(hi, shi[w]); }
  }
}

// lo/hi of row r of batch b: min/max over cols of A[b*s_batch + r*s_row + c*s_col];
// written to lo[b*out_sb + r], hi[b*out_sb + r]
__global__ void k_minmax_rows(const double* __restrict__ A, long long rows, long long cols,
                              long long s_row, long long s_col, long long s_batch,
                              double* lo_out, double* hi_out, long long out_sb) {
  const long long r = blockIdx.x, b = blockIdx.y;
  const double* a = A + b * s_batch + r * s_row;
  double lo = INFINITY, hi = -INFINITY;
  for (long long c = threadIdx.x; c < cols; c += blockDim.x) {
    double v = a[c * s_col];
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  block_minmax(lo, hi);
  if (threadIdx.x == 0) {
    lo_out[b * out_sb + r] = lo;
    hi_out[b * out_sb + r] = hi;
  }
}

void minmax_rows_out(const double* A, long long rows, long long cols, long long s_row,
                     long long s_col, int batch, long long s_batch, double* lo, double* hi,
                     long long out_sb, cudaStream_t s, Launches& L) {
  dim3 grid((unsigned)rows, (unsigned)batch);
  k_minmax_rows<<<grid, 256, 0, s>>>(A, rows, cols, s_row, s_col, s_batch, lo, hi, out_sb);
  L.add(1);
}

__global__ void k_anchor_minmax(const double* __restrict__ X, const int32_t* __restrict__ anchors,
                                int n_c, int F, double* lo_out, double* hi_out, long long out_sb) {
  const int c = blockIdx.x;
  const long long W = 3LL * F;
  double lo = INFINITY, hi = -INFINITY;
  for (long long e = threadIdx.x; e < (long long)n_c * F; e += blockDim.x) {
    long long a = e / F, f = e % F;
    double v = X[(long long)anchors[a] * W + (long long)c * F + f];
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  block_minmax(lo, hi);
  if (threadIdx.x == 0) {
    if (n_c == 0) { lo = 0.0; hi = 0.0; }
    lo_out[c * out_sb] = lo;
    hi_out[c * out_sb] = hi;
  }
}

void anchor_minmax_out(const double* X, const int32_t* anchors, int n_c, int F, double* lo,
                       double* hi, long long out_sb, cudaStream_t s, Launches& L) {
  k_anchor_minmax<<<3, 256, 0, s>>>(X, anchors, n_c, F, lo, hi, out_sb);
  L.add(1);
}

// ------------------------------------------------------------ header
struct HeaderArgs {
  long long total, anchors_off;
  long long coord_off[3];
  long long pad_at[10];   // byte offsets of 4-byte zero pads
  int n_pads;
  int n, F, k, n_c, cb, db, ab, kind;
};

__global__ void k_write_header(uint8_t* out, HeaderArgs h, const int32_t* __restrict__ anchors,
                               const double* __restrict__ qparams) {
  const int P = 4 * h.k + 2;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    uint32_t* w = (uint32_t*)out;
    w[0] = 0x31434D44u;  // "DMC1" little-endian
    w[1] = 1u;
    w[2] = (uint32_t)h.n;
    w[3] = (uint32_t)h.F;
    w[4] = (uint32_t)h.k;
    w[5] = (uint32_t)h.n_c;
    out[24] = (uint8_t)h.cb;
    out[25] = (uint8_t)h.db;
    out[26] = (uint8_t)h.ab;
    out[27] = (uint8_t)h.kind;
    w[7] = 64u;
    *(unsigned long long*)(out + 32) = (unsigned long long)h.total;
    for (int i = 40; i < 64; ++i) out[i] = 0;
    for (int i = 0; i < h.n_pads; ++i) *(uint32_t*)(out + h.pad_at[i]) = 0u;
  }
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  int32_t* ao = (int32_t*)(out + h.anchors_off);
  for (long long i = tid; i < h.n_c; i += nth) ao[i] = anchors[i];
  for (long long e = tid; e < 3LL * P; e += nth) {
    long long c = e / P, j = e % P;
    ((double*)(out + h.coord_off[c]))[j] = qparams[e];
  }
}

void write_header(uint8_t* out, const EncodeLayout& lay, const int32_t* anchors,
                  const double* qparams, cudaStream_t s, Launches& L) {
  HeaderArgs h{};
  h.total = lay.total;
  h.anchors_off = lay.anchors_off;
  for (int c = 0; c < 3; ++c) h.coord_off[c] = lay.coord_off[c];
  h.n_pads = 0;
  if (lay.n_c % 2) h.pad_at[h.n_pads++] = lay.anchors_off + 4LL * lay.n_c;
  for (int c = 0; c < 3; ++c) {
    const Section* secs[3] = {&lay.dict[c], &lay.coef[c], &lay.anch[c]};
    for (const Section* S : secs) {
      if (S->bits == 0) continue;
      long long wbytes = packed_words(S->count, S->bits) * 4;
      if (wbytes % 8) h.pad_at[h.n_pads++] = S->offset + wbytes;
    }
  }
  h.n = lay.n; h.F = lay.F; h.k = lay.k; h.n_c = lay.n_c;
  h.cb = lay.cb; h.db = lay.db; h.ab = lay.ab; h.kind = lay.kind;
  k_write_header<<<16, 256, 0, s>>>(out, h, anchors, qparams);
  L.add(1);
}

// ------------------------------------------------------------ quantize + pack
struct PackTask {
  long long groups;     // warp tasks in this section
  long long count;      // symbols
  long long offset;     // byte offset in the stream
  int bits;
  int type;             // 0 dictionary, 1 coefficients, 2 anchors
  int c;                // coordinate
};
struct PackTable {
  PackTask t[9];
  long long start[10];  // prefix of groups
  int n, F, k, n_c;
};

__device__ __forceinline__ long long quant_symbol(double x, double lo, double hi, int bits) {
  const double levels = (double)((1u << bits) - 1u);
  const double range = __dsub_rn(hi, lo);
  const double scale = range > 0.0 ? __ddiv_rn(levels, range) : 0.0;
  double t = __dmul_rn(__dsub_rn(x, lo), scale);
  double s = floor(__dadd_rn(t, 0.5));
  s = fmin(fmax(s, 0.0), levels);
  return (long long)s;
}

__device__ __forceinline__ void task_value(const PackTable& T, const PackTask& tk, long long idx,
                                           const double* U, const double* C, const double* X,
                                           const int32_t* anchors, const double* qparams,
                                           double& x, double& lo, double& hi) {
  const int k = T.k, F = T.F, n = T.n;
  const double* qp = qparams + (long long)tk.c * (4 * k + 2);
  if (tk.type == 0) {          // dictionary: idx = j*F + f -> U_c[f][j]
    long long j = idx / F, f = idx % F;
    x = U[((long long)tk.c * F + f) * k + j];
    lo = qp[j];
    hi = qp[k + j];
  } else if (tk.type == 1) {   // coefficients: idx = r*n + i -> C_c[r][i]
    long long r = idx / n;
    x = C[(long long)tk.c * k * n + idx];
    lo = qp[2 * k + r];
    hi = qp[3 * k + r];
  } else {                     // anchors: idx = a*F + f -> X[anchor a][c*F + f]
    long long a = idx / F, f = idx % F;
    x = X[(long long)anchors[a] * (3LL * F) + (long long)tk.c * F + f];
    lo = qp[4 * k];
    hi = qp[4 * k + 1];
  }
}

__global__ void __launch_bounds__(256) k_quant_pack(uint8_t* out, PackTable T,
                                                    const double* __restrict__ U,
                                                    const double* __restrict__ C,
                                                    const double* __restrict__ X,
                                                    const int32_t* __restrict__ anchors,
                                                    const double* __restrict__ qparams) {
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long total = T.start[9];
  for (long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
    int si = 0;
    while (si < 8 && w >= T.start[si + 1]) ++si;
    const PackTask tk = T.t[si];
    const long long g = w - T.start[si];
    const long long idx = g * 32 + lane;
    double x = 0.0, lo = 0.0, hi = 0.0;
    if (idx < tk.count) task_value(T, tk, idx, U, C, X, anchors, qparams, x, lo, hi);
    if (tk.bits == 0) {
      if (idx < tk.count) ((double*)(out + tk.offset))[idx] = x;
      continue;
    }
    unsigned s = (idx < tk.count) ? (unsigned)quant_symbol(x, lo, hi, tk.bits) : 0u;
    unsigned mine = 0;
    for (int j = 0; j < tk.bits; ++j) {
      unsigned word = __ballot_sync(0xffffffffu, (s >> j) & 1u);
      if (lane == j) mine = word;
    }
    if (lane < tk.bits) ((uint32_t*)(out + tk.offset))[g * tk.bits + lane] = mine;
  }
}

static PackTable make_table(const EncodeLayout& lay) {
  PackTable T{};
  T.n = lay.n; T.F = lay.F; T.k = lay.k; T.n_c = lay.n_c;
  int i = 0;
  T.start[0] = 0;
  for (int c = 0; c < 3; ++c) {
    const Section* secs[3] = {&lay.dict[c], &lay.coef[c], &lay.anch[c]};
    for (int ty = 0; ty < 3; ++ty) {
      const Section* S = secs[ty];
      PackTask& tk = T.t[i];
      tk.count = S->count;
      tk.offset = S->offset;
      tk.bits = S->bits;
      tk.type = ty;
      tk.c = c;
      tk.groups = (S->count + 31) / 32;
      T.start[i + 1] = T.start[i] + tk.groups;
      ++i;
    }
  }
  return T;
}

void quant_pack_sections(uint8_t* out, const EncodeLayout& lay, const double* U, const double* C,
                         const double* X, const int32_t* anchors, const double* qparams,
                         cudaStream_t s, Launches& L) {
  PackTable T = make_table(lay);
  long long warps = T.start[9];
  int grid = (int)std::min<long long>((warps * 32 + 255) / 256, 152 * 32);
  if (grid < 1) grid = 1;
  k_quant_pack<<<grid, 256, 0, s>>>(out, T, U, C, X, anchors, qparams);
  L.add(1);
}

// ------------------------------------------------------------ unpack
__global__ void __launch_bounds__(256) k_unpack(const uint8_t* __restrict__ in, PackTable T,
                                                double* __restrict__ Udeq,
                                                double* __restrict__ Cdeq,
                                                double* __restrict__ Ahat,
                                                const long long coord_off0,
                                                const long long coord_off1,
                                                const long long coord_off2) {
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long total = T.start[9] * 32;
  const int k = T.k, F = T.F, n = T.n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += nth) {
    long long w = e >> 5;
    int si = 0;
    while (si < 8 && w >= T.start[si + 1]) ++si;
    const PackTask tk = T.t[si];
    const long long idx = (w - T.start[si]) * 32 + (e & 31);
    if (idx >= tk.count) continue;
    const long long coff = tk.c == 0 ? coord_off0 : (tk.c == 1 ? coord_off1 : coord_off2);
    const double* qp = (const double*)(in + coff);
    double lo, hi;
    if (tk.type == 0) { long long j = idx / F; lo = qp[j]; hi = qp[k + j]; }
    else if (tk.type == 1) { long long r = idx / n; lo = qp[2 * k + r]; hi = qp[3 * k + r]; }
    else { lo = qp[4 * k]; hi = qp[4 * k + 1]; }
    double x;
    if (tk.bits == 0) {
      x = ((const double*)(in + tk.offset))[idx];
    } else {
      const uint32_t* wd = (const uint32_t*)(in + tk.offset) + (idx >> 5) * tk.bits;
      const int l = (int)(idx & 31);
      unsigned s = 0;
      for (int j = 0; j < tk.bits; ++j) s |= ((wd[j] >> l) & 1u) << j;
      const double levels = (double)((1u << tk.bits) - 1u);
      const double step = __ddiv_rn(__dsub_rn(hi, lo), levels);
      x = __dadd_rn(lo, __dmul_rn((double)s, step));
    }
    if (tk.type == 0) {
      long long j = idx / F, f = idx % F;
      Udeq[((long long)tk.c * F + f) * k + j] = x;
    } else if (tk.type == 1) {
      Cdeq[(long long)tk.c * k * n + idx] = x;
    } else {
      Ahat[(long long)tk.c * T.n_c * F + idx] = x;
    }
  }
}

__global__ void k_copy_anchors(const uint8_t* __restrict__ in, long long off, int n_c, int n,
                               int32_t* anchors, uint32_t* status) {
  const int32_t* a = (const int32_t*)(in + off);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_c;
       i += (long long)gridDim.x * blockDim.x) {
    int v = a[i];
    anchors[i] = v;
    if (v < 0 || v >= n || (i > 0 && a[i - 1] >= v)) atomicOr(status, ST_BITSTREAM);
  }
}

void unpack_sections(const uint8_t* in, const EncodeLayout& lay, double* Udeq, double* Cdeq,
                     double* Ahat, int32_t* anchors, double* /*qparams*/, uint32_t* status,
                     cudaStream_t s, Launches& L) {
  PackTable T = make_table(lay);
  if (lay.n_c > 0) {
    k_copy_anchors<<<(lay.n_c + 255) / 256, 256, 0, s>>>(in, lay.anchors_off, lay.n_c, lay.n,
                                                         anchors, status);
    L.add(1);
  }
  long long total = T.start[9] * 32;
  int grid = (int)std::min<long long>((total + 255) / 256, 152 * 32);
  if (grid < 1) grid = 1;
  k_unpack<<<grid, 256, 0, s>>>(in, T, Udeq, Cdeq, Ahat,
                                lay.coord_off[0], lay.coord_off[1], lay.coord_off[2]);
  L.add(1);
}

}  // namespace mc
