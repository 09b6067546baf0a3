// Adjacency build that allocates nothing (mesh_codec_adjacency_static).
//
// Some callers cannot call cudaMalloc at the point where they need a mesh's
// adjacency: real-time hosts that make every allocation before their loop
// starts (an allocation can block for milliseconds and may synchronise the
// device), and plug-ins inside a process whose device memory belongs to
// another framework's caching allocator (a cudaMalloc beside it can fail
// or fragment the pool that framework manages).  For them this entry point
// builds the same CSR adjacency as mesh_codec_create, with its temporary
// buffers in a file-scope device array instead of allocated memory.  The
// caller still provides the triangles and the three outputs.  The call
// waits for its stream once, to read the entry count and the error word.
//
// The scratch array below is part of the library image: every GPU on which
// the library is loaded holds it (7,865,344 bytes) until the process exits.
// All calls share it, so calls whose GPU work overlaps (different host
// threads, or different streams without ordering between them) race on it.
#include <cuda.h>

#include <mutex>

#include "mc_internal.cuh"

using namespace mc;

namespace {

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

constexpr int kMaxV = MESH_CODEC_STATIC_MAX_VERTICES;
constexpr int kMaxT = MESH_CODEC_STATIC_MAX_TRIANGLES;
// carve of the scratch array: status word, per-vertex raw degrees, raw row
// offsets, fill cursors, the raw (duplicated) neighbour lists, scan partials
constexpr size_t kOffStatus = 0;
constexpr size_t kOffRawDeg = align256(kOffStatus + 16);
constexpr size_t kOffRawOff = align256(kOffRawDeg + 4ull * kMaxV);
constexpr size_t kOffCursor = align256(kOffRawOff + 4ull * (kMaxV + 1));
constexpr size_t kOffRawCol = align256(kOffCursor + 4ull * kMaxV);
constexpr size_t kOffScan = align256(kOffRawCol + 4ull * 6 * kMaxT);
constexpr size_t kScratchBytes = align256(kOffScan + 4ull * (kMaxV / 2048 + 2));

static_assert(kScratchBytes == 7865344, "scratch size is documented in mesh_codec.h");

__device__ __align__(256) unsigned char g_adjacency_scratch[kScratchBytes];

// Device address of g_adjacency_scratch.  In host code the symbol's name is
// only a host-side handle; the address is looked up with cudaGetSymbolAddress
// with the device current, once per device and CUDA context: the module is
// loaded again in a new context (after cudaDeviceReset, or in another
// driver-API context on the same device) and the array can then move, so
// the cache is keyed on the context's unique ID.  Where the driver's context
// calls cannot be reached, the address is looked up on every call.
constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};
unsigned long long g_ctx_id[kMaxDevices] = {0};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// the current context's unique ID, or 0 when it cannot be read
unsigned long long current_context_id() {
  static std::once_flag once;
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = (CtxGetCurrentFn)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)p;
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

mesh_codec_status_t scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return MC_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return MC_E_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long id = current_context_id();
  if (id == 0 || !g_addr[dev] || g_ctx_id[dev] != id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_adjacency_scratch) != cudaSuccess || !p) return MC_E_CUDA;
    // the lookup made the device's primary context current if none was
    g_addr[dev] = p;
    g_ctx_id[dev] = id ? id : current_context_id();
  }
  *out = g_addr[dev];
  return MC_OK;
}

mesh_codec_status_t from_bits(uint32_t bits) {
  if (bits & (ST_BAD_INDEX | ST_DEGENERATE)) return MC_E_BAD_MESH;
  if (bits & ST_ISOLATED) return MC_E_ISOLATED_VERTEX;
  return MC_OK;
}

}  // namespace

extern "C" mesh_codec_status_t mesh_codec_adjacency_static(const int32_t* triangles,
                                                           int n_triangles, int n_vertices,
                                                           int32_t* row_ptr, int32_t* col_idx,
                                                           size_t col_idx_capacity,
                                                           int32_t* deg, int32_t* nnz_out,
                                                           void* stream) {
  if (!triangles || !row_ptr || !col_idx || !deg || !nnz_out) return MC_E_INVALID_ARG;
  if (n_vertices < 1 || n_triangles < 1) return MC_E_INVALID_ARG;
  if (n_vertices > kMaxV || n_triangles > kMaxT) return MC_E_INVALID_ARG;
  void* base = nullptr;
  mesh_codec_status_t st = scratch_address(&base);
  if (st != MC_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  char* b = (char*)base;
  uint32_t* status = (uint32_t*)(b + kOffStatus);
  CsrBuildTmp t{};
  t.raw_deg = (int32_t*)(b + kOffRawDeg);
  t.raw_off = (int32_t*)(b + kOffRawOff);
  t.cursor = (int32_t*)(b + kOffCursor);
  t.raw_col = (int32_t*)(b + kOffRawCol);
  t.scan_tmp = (int32_t*)(b + kOffScan);
  Launches L{nullptr};
  // the status word keeps the previous call's bits: clear it (the degree
  // counters and cursors are cleared by the build itself)
  if (cudaMemsetAsync(status, 0, 16, s) != cudaSuccess) return MC_E_CUDA;
  build_csr(triangles, n_triangles, n_vertices, t, row_ptr, nullptr, deg, status, s, L);
  uint32_t bits = 0;
  int32_t nnz = 0;
  if (cudaMemcpyAsync(&bits, status, sizeof(bits), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&nnz, row_ptr + n_vertices, sizeof(nnz), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MC_E_CUDA;
  st = from_bits(bits);
  if (st != MC_OK) return st;
  *nnz_out = nnz;
  if ((size_t)nnz > col_idx_capacity) return MC_E_BUFFER_TOO_SMALL;
  compact_csr(t, row_ptr, col_idx, n_vertices, s, L);
  if (cudaGetLastError() != cudaSuccess) return MC_E_CUDA;
  return MC_OK;
}
