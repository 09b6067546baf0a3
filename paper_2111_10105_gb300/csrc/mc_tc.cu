// Tensor-core GEMM for sm_103a: tcgen05.mma with TMA-fed shared memory and a
// TMEM accumulator.  It serves the mixed-precision forms of the codec's
// dense products: the two products of an orthogonal-iteration sweep
// (A_c^T Q and A_c W, Algorithm 1 / Eq. 7), the projection of Eq. 9 and the
// back-projection of Eq. 11.
//
// Shape: D (M x N, FP32 accumulate) = A (M x K) * B^T, both operands stored
// K-major ("TN"): A as rows of K elements, B as N rows of K elements.  One CTA
// computes a 128 x BN tile (BN a multiple of 16, <= 256) over a range of K
// (split-K across gridDim.z), with
//   warp 0 lane 0: TMA producer (cp.async.bulk.tensor, 128-byte swizzle),
//   warp 1 lane 0: MMA issuer (tcgen05.mma, kind::tf32 or kind::f16 bf16),
//   warps 0-3:     epilogue (tcgen05.ld from TMEM, FP32 -> global).
// A 4-stage ring of (A, B) chunks of 128 bytes of K per row is guarded by
// mbarriers (full: TMA bytes landed; empty: the MMAs that read the stage have
// completed, signalled by tcgen05.commit).  Every wait is bounded by a
// %globaltimer deadline (the process-wide limit of mesh_codec_set_wait_limit,
// 2 s by default); on timeout the CTA records an error bit, waits (bounded)
// for the copies it issued and for the products already issued to the tensor
// core, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "mc_internal.cuh"

namespace mc {
namespace tc {

constexpr int kBM = 128;
constexpr int kStages = 4;
constexpr uint32_t kAtomBytes = 128;            // one swizzled row of K
constexpr uint32_t kABytes = kBM * kAtomBytes;  // 16 KiB per stage
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s: default limit, and the drain's
std::atomic<unsigned long long> g_wait_ns{0};           // 0: kWaitNs

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
      " selp.b32 %0, 1, 0, P;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          unsigned long long deadline) {
  while (!mbar_try(bar, parity)) {
    if (gtimer() > deadline) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // SWIZZLE_128B
  return d;
}
// instruction descriptor: FP32 accumulator, K-major A and B, M = 128, N
__host__ __device__ constexpr uint32_t make_idesc(int fmt, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(kBM >> 4) << 24);
}

struct Args {
  int M, N, K;
  int BN, tmem_cols;
  int batch, splits, chunks_per_split, total_chunks;
  void* out;
  int out_kind;   // 0 fp32, 1 fp32 rounded to tf32, 2 bf16, 3 fp64, 4 fp64 added to out
  long long s0, s1, sb, split_stride;
  uint32_t* status;
  unsigned long long wait_ns;   // limit of every pipeline wait
};

template <int KIND>  // 0: tf32 (4-byte elements), 1: bf16
__global__ void __launch_bounds__(128, 1) k_umma_tn(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB,
                                                    Args a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t b_bytes = (uint32_t)a.BN * kAtomBytes;
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kABytes;
  uint64_t* bars = (uint64_t*)(sB + kStages * b_bytes);  // full[4], empty[4], done
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * kStages + 1);
  int* abort_flag = (int*)(tmem_slot + 1);
  int* issued_slot = abort_flag + 1;   // chunks whose copies the producer issued
  int* consumed_slot = abort_flag + 2; // chunks whose products the issuer committed
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * kStages,
                 done = full0 + 16 * kStages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int zb = blockIdx.z, b = zb % a.batch, split = zb / a.batch;
  const int n0 = blockIdx.x * a.BN, m0 = blockIdx.y * kBM;
  const int kc0 = split * a.chunks_per_split;
  const int nk = min(a.total_chunks, kc0 + a.chunks_per_split) - kc0;
  constexpr int atom_elems = KIND == 0 ? 32 : 64;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    *issued_slot = 0;
    *consumed_slot = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const unsigned long long deadline = gtimer() + a.wait_ns;

  if (warp == 0 && lane == 0 && nk > 0) {
    // producer
    int i = 0;
    for (; i < nk; ++i) {
      const int s = i % kStages;
      if (i >= kStages) {
        if (!mbar_wait(empty0 + 8 * s, ((i / kStages) - 1) & 1, deadline)) {
          *abort_flag = 1;
          break;
        }
      }
      if (*(volatile int*)abort_flag) break;
      const int kel = (kc0 + i) * atom_elems;
      mbar_expect_tx(full0 + 8 * s, kABytes + b_bytes);
      tma_load_3d(smem_u32(sA + s * kABytes), &tmA, kel, m0, b, full0 + 8 * s);
      tma_load_3d(smem_u32(sB + s * b_bytes), &tmB, kel, n0, b, full0 + 8 * s);
    }
    *issued_slot = i;
  } else if (warp == 1 && lane == 0 && nk > 0) {
    // MMA issuer
    const uint32_t idesc = make_idesc(KIND == 0 ? 2 : 1, a.BN);
    int i = 0;
    for (; i < nk; ++i) {
      const int s = i % kStages;
      if (!mbar_wait(full0 + 8 * s, (i / kStages) & 1, deadline)) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t aa = smem_u32(sA + s * kABytes), bb = smem_u32(sB + s * b_bytes);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint64_t da = sw128_desc(aa + 32 * j), db = sw128_desc(bb + 32 * j);
        const uint32_t acc = (i > 0 || j > 0) ? 1u : 0u;
        if (KIND == 0) {
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc)
              : "memory");
        } else {
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              empty0 + 8 * s)
          : "memory");
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done)
        : "memory");
    *consumed_slot = i;
  }
  __syncwarp();
  // epilogue: every thread owns one accumulator row
  bool ok = nk > 0 && mbar_wait(done, 0, deadline + a.wait_ns);
  ok = __syncthreads_and(ok && !*(volatile int*)abort_flag) != 0;   // CTA-uniform
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = warp * 32 + lane, m = m0 + row;
    const long long base = (long long)b * a.sb + (long long)split * a.split_stride;
    for (int c = 0; c < a.BN; c += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
          "%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < a.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c + j;
          if (n < a.N) {
            const long long o = base + (long long)m * a.s0 + (long long)n * a.s1;
            const float v = __uint_as_float(r[j]);
            if (a.out_kind == 0) {
              ((float*)a.out)[o] = v;
            } else if (a.out_kind == 1) {
              uint32_t t;
              asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
              ((float*)a.out)[o] = __uint_as_float(t);
            } else if (a.out_kind == 2) {
              ((__nv_bfloat16*)a.out)[o] = __float2bfloat16_rn(v);
            } else if (a.out_kind == 3) {
              ((double*)a.out)[o] = (double)v;
            } else {   // one thread per element (no K split): a plain read-modify-write
              ((double*)a.out)[o] += (double)v;
            }
          }
        }
      }
    }
  }
  if (!ok) {
    if (threadIdx.x == 0 && nk > 0) atomicOr(a.status, ST_TC_TIMEOUT);
    // drain before TMEM and shared memory are released: wait (bounded by the
    // default limit) for the last copy issued into every stage, and for the
    // products issued to the tensor core (the issuer committed them all to
    // `done`, also when it stopped early)
    if (warp == 0 && lane == 0 && nk > 0) {
      const unsigned long long d2 = gtimer() + kWaitNs;
      const int issued = *(volatile int*)issued_slot;
      for (int s = 0; s < kStages && s < issued; ++s) {
        const int last = s + kStages * ((issued - 1 - s) / kStages);   // last chunk in stage s
        mbar_wait(full0 + 8 * s, (last / kStages) & 1, d2);
      }
      mbar_wait(done, 0, d2);
      // and for the arrivals of the per-stage commits of the products
      const int consumed = *(volatile int*)consumed_slot;
      for (int s = 0; s < kStages && s < consumed; ++s) {
        const int last = s + kStages * ((consumed - 1 - s) / kStages);
        mbar_wait(empty0 + 8 * s, (last / kStages) & 1, d2);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols)
                 : "memory");
  }
}

// ------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

}  // namespace tc

// rows x K operand (K innermost, `pitch` elements between rows, `bpitch` between
// batches), boxes of 128 bytes of K x box_rows rows, 128-byte swizzle
bool tc_operand_map(void* map_out, const void* base, int elem_bytes, long long K, long long rows,
                    int batch, long long pitch, long long bpitch, int box_rows) {
  tc::EncodeTiledFn fn = tc::encode_fn();
  if (!fn) return false;
  if (((uintptr_t)base & 15) || (pitch * elem_bytes) % 16 || (bpitch * elem_bytes) % 16)
    return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)(pitch * elem_bytes), (cuuint64_t)(bpitch * elem_bytes)};
  cuuint32_t box[3] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn((CUtensorMap*)map_out,
                  elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                  3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t tc_smem_bytes(int BN) {
  return 1024 + (size_t)tc::kStages * (tc::kABytes + (size_t)BN * tc::kAtomBytes) + 256;
}

// D = A B^T with FP32 accumulation; out element (m, n) of batch b / split z at
// out + b*sb + z*split_stride + m*s0 + n*s1.  kind: 0 tf32, 1 bf16.
// Returns the number of K splits used (each writes its own partial).
int umma_tn(int kind, const void* mapA, const void* mapB, int M, int N, int K, int batch,
            int splits, void* out, int out_kind, long long s0, long long s1, long long sb,
            long long split_stride, uint32_t* status, cudaStream_t s, Launches& L) {
  const int atom = kind == 0 ? 32 : 64;
  int BN = N <= 256 ? ((N + 15) / 16) * 16 : 256;
  int cols = 32;
  while (cols < BN) cols <<= 1;
  tc::Args a{};
  a.M = M; a.N = N; a.K = K; a.BN = BN; a.tmem_cols = cols; a.batch = batch;
  a.total_chunks = (K + atom - 1) / atom;
  if (splits < 1) splits = 1;
  a.chunks_per_split = (a.total_chunks + splits - 1) / splits;
  a.splits = (a.total_chunks + a.chunks_per_split - 1) / a.chunks_per_split;
  a.out = out; a.out_kind = out_kind; a.s0 = s0; a.s1 = s1; a.sb = sb; a.split_stride = split_stride;
  a.status = status;
  const unsigned long long lim = tc::g_wait_ns.load(std::memory_order_relaxed);
  a.wait_ns = lim ? lim : tc::kWaitNs;
  const size_t sm = tc_smem_bytes(BN);
  dim3 grid((N + BN - 1) / BN, (M + tc::kBM - 1) / tc::kBM, batch * a.splits);
  const CUtensorMap& ma = *(const CUtensorMap*)mapA;
  const CUtensorMap& mb = *(const CUtensorMap*)mapB;
  if (kind == 0) {
    cudaFuncSetAttribute(tc::k_umma_tn<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    tc::k_umma_tn<0><<<grid, 128, sm, s>>>(ma, mb, a);
  } else {
    cudaFuncSetAttribute(tc::k_umma_tn<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    tc::k_umma_tn<1><<<grid, 128, sm, s>>>(ma, mb, a);
  }
  L.add(1);
  return a.splits;
}

// ------------------------------------------------------------ operand packing
// dst[b][r][c] (pitch dpitch, batch pitch dbp) = round(src(b, r, c)) for
// r < rows, c < cols, zero for cols <= c < dcols; src element at
// src[b*ssb + r*sr + c*sc].  kind 0: FP32 rounded to TF32 (nearest, ties
// away, as cvt.rna.tf32.f32), kind 1: BF16 (nearest even).
template <typename S>
__global__ void k_pack_operand(const S* __restrict__ src, long long ssb, long long sr,
                               long long sc, int batch, long long rows, long long cols,
                               long long dcols, long long dpitch, long long dbp, int kind,
                               void* dst) {
  const long long total = (long long)batch * rows * dcols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long b = e / (rows * dcols), rem = e % (rows * dcols);
    long long r = rem / dcols, c = rem % dcols;
    float v = 0.f;
    if (c < cols) v = (float)src[b * ssb + r * sr + c * sc];
    long long o = b * dbp + r * dpitch + c;
    if (kind == 0) {
      uint32_t t;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
      ((float*)dst)[o] = __uint_as_float(t);
    } else {
      ((__nv_bfloat16*)dst)[o] = __float2bfloat16_rn(v);
    }
  }
}

void pack_operand_f64(const double* src, long long ssb, long long sr, long long sc, int batch,
                      long long rows, long long cols, long long dcols, long long dpitch,
                      long long dbp, int kind, void* dst, cudaStream_t s, Launches& L) {
  long long total = (long long)batch * rows * dcols;
  int g = (int)std::min<long long>((total + 255) / 256, 152 * 32);
  k_pack_operand<double><<<std::max(g, 1), 256, 0, s>>>(src, ssb, sr, sc, batch, rows, cols,
                                                        dcols, dpitch, dbp, kind, dst);
  L.add(1);
}

void pack_operand_f32(const float* src, long long ssb, long long sr, long long sc, int batch,
                      long long rows, long long cols, long long dcols, long long dpitch,
                      long long dbp, int kind, void* dst, cudaStream_t s, Launches& L) {
  long long total = (long long)batch * rows * dcols;
  int g = (int)std::min<long long>((total + 255) / 256, 152 * 32);
  k_pack_operand<float><<<std::max(g, 1), 256, 0, s>>>(src, ssb, sr, sc, batch, rows, cols, dcols,
                                                       dpitch, dbp, kind, dst);
  L.add(1);
}

// out[e] = sum over z < splits of part[z*stride + e] (fixed order), as FP64
__global__ void k_sum_splits(const float* __restrict__ part, int splits, long long stride,
                             long long count, double* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += (double)part[z * stride + e];
    out[e] = s;
  }
}

void sum_splits(const float* part, int splits, long long stride, long long count, double* out,
                cudaStream_t s, Launches& L) {
  int g = (int)std::min<long long>((count + 255) / 256, 152 * 8);
  k_sum_splits<<<std::max(g, 1), 256, 0, s>>>(part, splits, stride, count, out);
  L.add(1);
}

}  // namespace mc

// ------------------------------------------------------------ self test
using namespace mc;

extern "C" mesh_codec_status_t mesh_codec_set_wait_limit(unsigned long long ns) {
  tc::g_wait_ns.store(ns, std::memory_order_relaxed);
  return MC_OK;
}

extern "C" mesh_codec_status_t mesh_codec_selftest_gemm(int kind, int M, int N, int K,
                                                        int splits, const float* A,
                                                        const float* B, double* C,
                                                        void* stream) {
  if ((kind != 0 && kind != 1) || M < 1 || N < 1 || K < 1 || !A || !B || !C) return MC_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int eb = kind == 0 ? 4 : 2;
  const long long Kp = ((K + 63) / 64) * 64;
  void *Ap = nullptr, *Bp = nullptr;
  float* part = nullptr;
  uint32_t* status = nullptr;
  Launches L{nullptr};
  mesh_codec_status_t st = MC_OK;
  int used = 1;
  alignas(64) unsigned char ma[128], mb[128];
  if (cudaMalloc(&Ap, (size_t)M * Kp * eb) != cudaSuccess ||
      cudaMalloc(&Bp, (size_t)N * Kp * eb) != cudaSuccess ||
      cudaMalloc(&part, sizeof(float) * (size_t)std::max(splits, 1) * M * N) != cudaSuccess ||
      cudaMalloc(&status, 16) != cudaSuccess) {
    st = MC_E_OOM;
    goto out;
  }
  cudaMemsetAsync(status, 0, 16, s);
  pack_operand_f32(A, 0, K, 1, 1, M, K, Kp, Kp, 0, kind, Ap, s, L);
  pack_operand_f32(B, 0, K, 1, 1, N, K, Kp, Kp, 0, kind, Bp, s, L);
  if (!tc_operand_map(ma, Ap, eb, Kp, M, 1, Kp, Kp * M, 128) ||
      !tc_operand_map(mb, Bp, eb, Kp, N, 1, Kp, Kp * N, N <= 256 ? ((N + 15) / 16) * 16 : 256)) {
    st = MC_E_CUDA;
    goto out;
  }
  used = umma_tn(kind, ma, mb, M, N, K, 1, splits, part, 0, N, 1, 0, (long long)M * N, status, s,
                 L);
  sum_splits(part, used, (long long)M * N, (long long)M * N, C, s, L);
  {
    uint32_t bits = 0;
    if (cudaMemcpyAsync(&bits, status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      st = MC_E_CUDA;
    else if (bits & ST_TC_TIMEOUT)
      st = MC_E_TIMEOUT;
    else if (bits)
      st = MC_E_CUDA;
  }
out:
  cudaStreamSynchronize(s);
  if (Ap) cudaFree(Ap);
  if (Bp) cudaFree(Bp);
  if (part) cudaFree(part);
  if (status) cudaFree(status);
  return st;
}
