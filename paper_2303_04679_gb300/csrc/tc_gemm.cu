// BF16 GEMM on the fifth-generation tensor cores (tcgen05), the dense
// contraction of the learned warm start (3-D convolutions as im2col GEMMs).
//
//   D[M x N] (+)= A[M x K] * B[N x K]^T      A, B: BF16, K contiguous (K-major)
//                                            accumulate: FP32 in tensor memory
//
// One CTA computes a 128 x BN tile of D over a range of K (split-K over
// blockIdx.z).  Four warps:
//   warp 0 lane 0  producer: TMA loads of 128 x 64 A and BN x 64 B tiles
//                  (128-byte swizzle) into a 4-stage shared-memory ring,
//                  completion counted on a "full" mbarrier per stage;
//   warp 1 lane 0  issues tcgen05.mma (M = 128, N = BN, K = 16, four per
//                  stage) from shared-memory descriptors into a TMEM
//                  accumulator of BN FP32 columns, and tcgen05.commit frees the
//                  stage ("empty" mbarrier) once its MMAs have read it;
//   all four warps epilogue: tcgen05.ld of the accumulator rows (warp w owns
//                  TMEM lanes 32w..32w+31 = tile rows), optional bias and
//                  ReLU, store as BF16 or FP32, or FP32 atomic add (split-K).
// Every mbarrier wait is bounded: on timeout the CTA records an error code,
// stops issuing work, waits (bounded) for the MMAs it issued, frees its TMEM
// and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_gemm.h"

namespace modil_tc {

constexpr int BM = 128, BK = 64, STAGES = 4, NTHREADS = 128;
constexpr long long kSpin = 1LL << 24;  // polls of one mbarrier wait before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < kSpin; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes (64 BF16), 8-row swizzle atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int BN>
struct Smem {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int BYTES = STAGES * STAGE + 1024 /* align */ + 256 /* barriers */;
};

template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
k_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, const GemmArgs g) {
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "MMA N");
  constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;  // TMEM columns: power of two >= 32
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * Smem<BN>::STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int nk_total = (g.K + BK - 1) / BK;
  // weight gradient of a convolution: blockIdx.z = tap * wsplits + split
  const int wtap = g.conv == 2 ? (int)blockIdx.z / g.wsplits : 0;
  const int kc0 = (g.conv == 2 ? (int)blockIdx.z - wtap * g.wsplits : (int)blockIdx.z) * g.kchunks;
  const int kc1 = min(nk_total, kc0 + g.kchunks);
  const int nk = max(0, kc1 - kc0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  int issued = 0;  // MMA issuer: 1 once a commit to "done" is outstanding

  if (nk > 0) {
    if (warp == 0 && lane == 0) {
      // producer
      for (int i = 0; i < nk; ++i) {
        const int s = i % STAGES, use = i / STAGES;
        if (use > 0 && !mbar_wait(empty + s, (use - 1) & 1)) {
          *abort_flag = 1;
          atomicCAS(g.err, 0, 1);
          break;
        }
        if (*abort_flag) break;
        unsigned char* st = smem + s * Smem<BN>::STAGE;
        mbar_expect_tx(full + s, Smem<BN>::STAGE);
        if (g.conv == 2) {
          // chunk -> its first voxel (x and y flattened: a y shift is an
          // offset of S, 16-byte aligned for S >= 8, and rows past the plane's
          // ends read as zero); the tap's x-shifted copy
          const int v0 = (kc0 + i) * BK, S = g.S, S2 = S * S;
          const int xy0 = v0 % S2, r2 = v0 / S2, z0 = r2 % S, b0 = r2 / S;
          const int dz = wtap / 9 - 1, dy = (wtap / 3) % 3 - 1, dx = wtap % 3 - 1;
          tma_load_4d(st, &ta, full + s, xy0 + dy * S, z0 + dz, b0, (dx + 1) * g.wC + m0);
          tma_load_2d(st + Smem<BN>::A_BYTES, &tb, full + s, v0, n0);
        } else if (g.conv) {
          // chunk -> (tap, channel block); the output tile's first voxel
          const int kc = kc0 + i, tap = kc / g.cc, c0 = (kc - tap * g.cc) * BK;
          const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
          const int S = g.S;
          const int x0 = m0 % S, r1 = m0 / S, y0 = r1 % S, r2 = r1 / S, z0 = r2 % S, b0 = r2 / S;
          tma_load_5d(st, &ta, full + s, c0, x0 + g.sign * dx, y0 + g.sign * dy, z0 + g.sign * dz, b0);
          if (g.b_tap_mid)
            tma_load_3d(st + Smem<BN>::A_BYTES, &tb, full + s, c0, tap, n0);
          else
            tma_load_3d(st + Smem<BN>::A_BYTES, &tb, full + s, c0, n0, tap);
        } else {
          const int kx = (kc0 + i) * BK;
          tma_load_2d(st, &ta, full + s, kx, m0);
          tma_load_2d(st + Smem<BN>::A_BYTES, &tb, full + s, kx, n0);
        }
      }
    } else if (warp == 1 && lane == 0) {
      // MMA issuer
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      for (int i = 0; i < nk; ++i) {
        const int s = i % STAGES, use = i / STAGES;
        if (!mbar_wait(full + s, use & 1)) {
          *abort_flag = 1;
          atomicCAS(g.err, 0, 2);
          break;
        }
        if (*abort_flag) break;
        fence_after();
        const uint32_t a = smem_u32(smem + s * Smem<BN>::STAGE);
        const uint32_t b = a + Smem<BN>::A_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
          mma_bf16(tmem, sw128_desc(a + 32 * k), sw128_desc(b + 32 * k), idesc, (i > 0 || k > 0) ? 1u : 0u);
        mma_commit(empty + s);
      }
      mma_commit(done);  // also tracks any MMAs issued before an abort
      issued = 1;
    }
  }
  __syncwarp();
  // epilogue (every warp: 32 accumulator rows each)
  bool ok = true;
  if (nk > 0) ok = mbar_wait(done, 0);
  if (!ok) atomicCAS(g.err, 0, 3);
  fence_after();
  if (nk > 0 && ok && !*abort_flag) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c = 0; c < BN; c += 16) {
      float v[16];
      tmem_ld16(trow + c, v);
      const int col = n0 + c;
      if (row >= g.M || col >= g.N) continue;
      const int ncol = min(16, g.N - col);
      if (g.mode == GEMM_STORE_BF16_MASK) {
        const __nv_bfloat16* a = static_cast<const __nv_bfloat16*>(g.act) + (long long)row * g.ldd + col;
        __nv_bfloat16* d = static_cast<__nv_bfloat16*>(g.D) + (long long)row * g.ldd + col;
        for (int j = 0; j < ncol; ++j) d[j] = __float2bfloat16_rn(__bfloat162float(a[j]) > 0.f ? v[j] : 0.f);
      } else if (g.mode == GEMM_STORE_BF16) {
        if (g.bias)
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] += (col + j < g.N) ? g.bias[col + j] : 0.f;
        if (g.relu)
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
        __nv_bfloat16* d = static_cast<__nv_bfloat16*>(g.D) + (long long)row * g.ldd + col;
        if (ncol == 16 && (g.ldd & 7) == 0) {
          __align__(16) __nv_bfloat162 h[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
          reinterpret_cast<uint4*>(d)[0] = reinterpret_cast<uint4*>(h)[0];
          reinterpret_cast<uint4*>(d)[1] = reinterpret_cast<uint4*>(h)[1];
        } else {
          for (int j = 0; j < ncol; ++j) d[j] = __float2bfloat16_rn(v[j]);
        }
      } else if (g.mode == GEMM_STORE_F32) {
        float* d = static_cast<float*>(g.D) + (long long)row * g.ldd + col;
        if (g.bias)
          for (int j = 0; j < ncol; ++j) v[j] += g.bias[col + j];
        if (ncol == 16 && (g.ldd & 3) == 0) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            reinterpret_cast<float4*>(d)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        } else {
          for (int j = 0; j < ncol; ++j) d[j] = v[j];
        }
      } else {  // GEMM_ATOMIC_F32 (weight gradients: rows of the tap)
        float* d = static_cast<float*>(g.D) + ((long long)wtap * g.wC + row) * g.ldd + col;
        for (int j = 0; j < ncol; ++j) atomicAdd(d + j, v[j]);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
  }
  (void)issued;
}

template <int BN>
static cudaError_t set_smem_attr() {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Smem<BN>::BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return cudaSuccess;
}

template <int BN>
static cudaError_t launch_bn(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, int splits,
                             cudaStream_t s) {
  const size_t smem = Smem<BN>::BYTES;
  cudaError_t e = set_smem_attr<BN>();
  if (e != cudaSuccess) return e;
  dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, splits);
  k_gemm<BN><<<grid, NTHREADS, smem, s>>>(ta, tb, g);
  return cudaGetLastError();
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiled encoder();

cudaError_t prepare_gemm() {
  if (!encoder()) return cudaErrorNotSupported;
  cudaError_t e = set_smem_attr<16>();
  if (e == cudaSuccess) e = set_smem_attr<32>();
  if (e == cudaSuccess) e = set_smem_attr<64>();
  if (e == cudaSuccess) e = set_smem_attr<128>();
  if (e == cudaSuccess) e = set_smem_attr<256>();
  return e;
}

cudaError_t launch_gemm(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, int bn, int splits,
                        cudaStream_t s) {
  switch (bn) {
    case 16: return launch_bn<16>(ta, tb, g, splits, s);
    case 32: return launch_bn<32>(ta, tb, g, splits, s);
    case 64: return launch_bn<64>(ta, tb, g, splits, s);
    case 128: return launch_bn<128>(ta, tb, g, splits, s);
    case 256: return launch_bn<256>(ta, tb, g, splits, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Tensor maps (driver entry point fetched through the runtime once)
// ---------------------------------------------------------------------------
static EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

// A row-major BF16 matrix of `rows` rows, `k` used columns and a row pitch of
// `ld` elements, as 64-column x box_rows tiles with 128-byte swizzle; reads
// past k or rows return zeros.
int make_kmajor_map(CUtensorMap* m, const void* base, long long rows, long long k, long long ld, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc) return -1;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 2) & 15) || k > ld) return -2;
  cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -3;
}

int make_act_map(CUtensorMap* m, const void* base, int C, int S, int B) {
  EncodeTiled enc = encoder();
  if (!enc) return -1;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (C % 8) || S < 8 || C > 65536) return -2;
  const int bx = S < BM ? S : BM, by = (BM / bx) < S ? BM / bx : S, bz = BM / (bx * by);
  if (bx * by * bz != BM || bz > S) return -2;
  const cuuint64_t cs = (cuuint64_t)C * 2;
  cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)S, (cuuint64_t)S, (cuuint64_t)S, (cuuint64_t)B};
  cuuint64_t strides[4] = {cs, cs * S, cs * S * S, cs * S * S * S};
  cuuint32_t box[5] = {(cuuint32_t)BK, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -3;
}

int make_shift3_map(CUtensorMap* m, const void* base, int C, int S, int B) {
  EncodeTiled enc = encoder();
  if (!enc) return -1;
  // x and y flattened into one axis of S^2 voxels, so that a K chunk is one
  // 64-voxel (128-byte) line: the 128B swizzle pattern assumes 128-byte rows
  if ((reinterpret_cast<uintptr_t>(base) & 15) || S < 8 || (S * S) % BK) return -2;
  const cuuint64_t ps = (cuuint64_t)S * S * 2;  // bytes of one z plane
  cuuint64_t dims[4] = {(cuuint64_t)S * S, (cuuint64_t)S, (cuuint64_t)B, (cuuint64_t)3 * C};
  cuuint64_t strides[3] = {ps, ps * S, ps * S * B};
  cuuint32_t box[4] = {(cuuint32_t)BK, 1, 1, (cuuint32_t)BM};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -3;
}

int make_3d_map(CUtensorMap* m, const void* base, long long d0, long long d1, long long d2, long long s1,
                long long s2, int b1, int b2) {
  EncodeTiled enc = encoder();
  if (!enc) return -1;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((s1 * 2) & 15) || ((s2 * 2) & 15)) return -2;
  cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
  cuuint64_t strides[2] = {(cuuint64_t)(s1 * 2), (cuuint64_t)(s2 * 2)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)b1, (cuuint32_t)b2};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -3;
}

}  // namespace modil_tc
