// mlp.cu -- the deformation MLP of Sec. 4 ("MLP") on the 5th-generation
// tensor cores: delta_x = MLP(gamma(x / d_u), gamma(t)), 8 hidden layers of
// 256 with ReLU, a linear head to the 3 offset components, forward and
// backward for B frames x N Gaussians (rows m = b N + g).
//
// Two kinds of kernel, both BF16 operands with FP32 accumulation in TMEM
// (tcgen05.mma issued by one elected thread, operand tiles in shared memory
// in the 128-byte swizzled layout, TMA loads completing on mbarriers):
//  * fused all-layer kernels over pairs of 128-row tiles per CTA (one CTA per
//    SM, the two tiles' accumulators filling TMEM, the epilogue of one tile
//    overlapping the MMAs of the other; a TMA warp streams the weights, an
//    MMA warp, 8 epilogue warps):
//      forward        every layer's output (bias, ReLU, BF16) written back
//                     into the tile as the next layer's operand; training:
//                     each tile also TMA-stored row-major (H_l, the encoding)
//                     and the ReLU masks as bits; inference: nothing kept
//      dZ chain       dZ_7 = (dZ_head W_head) * mask_7, ..., dZ_0, then
//                     d(encoding) = dZ_0 W_0 (FP32), each dZ tile TMA-stored
//                     row-major
//  * a tiled GEMM (TMA pipeline, 4 epilogue warps), for the weight gradients
//    dW_l = dZ_l^T H_{l-1}: the batch rows are the reduction dimension, so
//    both operands are read MN-major straight from the row-major dZ_l and
//    H_{l-1} (transpose bits of the instruction descriptor), the 256 output
//    rows as two M = 128 accumulators sharing each B tile, partial sums per
//    share of rows reduced afterwards; its epilogue warps, idle during the
//    main loop, sum dZ_l's columns (the bias gradient) from each stage.  The
//    same GEMM with other epilogues runs the one-GEMM-per-layer forward and
//    dZ chain, kept as a test mode the fused kernels are checked against.
// Waits on mbarriers are bounded (about 2 s): a wait that runs out records
// GFTORF_ERR_TIMEOUT in the status word and the CTA winds down.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "gftorf_internal.cuh"

namespace gftorf {
namespace {

constexpr int kW = GFTORF_MLP_WIDTH;    // 256
constexpr int kDepth = GFTORF_MLP_DEPTH;  // 8
constexpr int kIn = GFTORF_MLP_INPUT;   // 128 (84 used)
constexpr int kFreq = 10;
constexpr int kHeadRows = 32;           // head padded to the MMA's N = 32
constexpr int kExt = 16;                // bias column (+ padding) after each dW block
constexpr int BM = 128, BK = 64;

enum Epi { EPI_HIDDEN = 0, EPI_HEAD = 1, EPI_MASK = 2, EPI_F32 = 3, EPI_ATOMIC = 4, EPI_PARTIAL = 5 };
constexpr int kMaxSplits = 192;  // row splits of a weight-gradient GEMM

struct GemmArgs {
  int kb_total;      // k-blocks (of 64) of the reduction
  int kb_per_split;  // k-blocks per CTA along gridDim.z
  int rows_valid;    // output rows that exist (epilogue guard)
  int cols_valid;    // output columns that exist
  const float* bias;
  __nv_bfloat16* out_b;   // row-major bf16 output (ld = ldo)
  int ldo;
  float* out_f;           // FP32 output (ld = ldf)
  int ldf;
  uint32_t* mbits;            // ReLU masks, one bit per unit, [rows][8] words:
                              // written by EPI_HIDDEN, read by EPI_MASK
  float* dbias;               // EPI_PARTIAL with an MN-major A: A's column sums over the
                              // CTA's rows (the bias gradient) added at dbias[n ldb]
  int ldb;
  int inject_no_loads;        // test hook: the producer issues nothing (waits run out)
  unsigned long long wait_ns; // limit of one mbarrier wait
  int* status;
};

// ---- PTX wrappers ----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase with the given parity to complete.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status,
                          unsigned long long limit_ns = 2000000000ull) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) {
      atomicExch(status, (int)GFTORF_ERR_TIMEOUT);
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}
// tile from shared memory to global memory (bulk async-group of this thread)
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int c0,
                                             int c1) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(src), "r"(c0), "r"(c1)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// this thread's bulk stores have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// ... and have completed
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
// K-major operand tile in shared memory, rows of 128 bytes with the 128-byte
// swizzle (8-row groups 1024 bytes apart); the start address may step along K
// inside the 128-byte row.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                             // leading offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;                   // stride between 8-row groups
  d |= (uint64_t)1 << 46;                             // descriptor version
  d |= (uint64_t)2 << 61;                             // 128-byte swizzle
  return d;
}
// MN-major operand tile (the M or N index contiguous): 64-element chunks of
// the MN index, each 8192 bytes (64 K-rows of 128 bytes, the 128-byte swizzle
// over 8-row groups 1024 bytes apart), as a TMA box of 64 x 64 lands them;
// the start address steps along K by whole 8-row groups.
__device__ __forceinline__ uint64_t sw128_mn_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)(8192 >> 4) << 16;                   // between 64-element MN chunks
  d |= (uint64_t)(1024 >> 4) << 32;                   // between 8-row K groups
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// kind::f16 instruction descriptor: BF16 x BF16 -> FP32; A and B K-major
// unless mn_a / mn_b (MN-major)
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n, int mn_a = 0, int mn_b = 0) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)mn_a << 15) | ((uint32_t)mn_b << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per lane)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 consecutive FP32 columns of this warp's 32 TMEM lanes: one load and one
// wait for twice the columns of tmem_ld32 (half the exposed load latency)
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float* v) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {"
      "%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
      "%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
      "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]),
        "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]),
        "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
        "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]),
        "=r"(r[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void store_row_bf16(__nv_bfloat16* dst, const float* v) {
  uint4 q[4];
  uint32_t* w = reinterpret_cast<uint32_t*>(q);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    w[i] = *reinterpret_cast<uint32_t*>(&h);
  }
  uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
  for (int i = 0; i < 4; ++i) d[i] = q[i];
}

// 32 columns [n, n + 32) of output row m
// bf16_rn(v) > 0 for v >= 0 (or -0): v above 2^-134, half the smallest BF16
// subnormal (ties round to even, i.e. to zero)
__device__ __forceinline__ uint32_t relu_bits(const float* v) {
  uint32_t bits = 0;
#pragma unroll
  for (int j = 0; j < 32; ++j) bits |= (v[j] > 0x1p-134f ? 1u : 0u) << j;
  return bits;
}

template <int EPI>
__device__ __forceinline__ void epilogue(const GemmArgs& p, int m, int n, float* v) {
  if (EPI == EPI_HIDDEN || EPI == EPI_MASK) {
    if (EPI == EPI_HIDDEN) {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j] + __ldg(p.bias + n + j), 0.f);
      p.mbits[(size_t)m * (kW / 32) + n / 32] = relu_bits(v);
    } else {
      const uint32_t bits = __ldg(p.mbits + (size_t)m * (kW / 32) + n / 32);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (!((bits >> j) & 1u)) v[j] = 0.f;
    }
    store_row_bf16(p.out_b + (size_t)m * p.ldo + n, v);
  } else if (EPI == EPI_HEAD) {
    if (m < p.rows_valid)
      for (int j = 0; j < 3; ++j) p.out_f[(size_t)m * 3 + j] = v[j] + __ldg(p.bias + j);
  } else if (EPI == EPI_F32) {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (n + j < p.cols_valid) p.out_f[(size_t)m * p.ldf + n + j] = v[j];
  } else if (EPI == EPI_PARTIAL) {  // this CTA's partial sum over its rows of the batch
    if (m < p.rows_valid && n < p.cols_valid) {
      float4* d = reinterpret_cast<float4*>(
          p.out_f + ((size_t)blockIdx.z * p.rows_valid + m) * p.ldf + n);
#pragma unroll
      for (int q = 0; q < 8; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
  } else {  // EPI_ATOMIC
    if (m < p.rows_valid) {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (n + j < p.cols_valid) atomicAdd(p.out_f + (size_t)m * p.ldf + n + j, v[j]);
    }
  }
}

// MT: M = 128 accumulators per CTA sharing each B tile (A tile of 128 MT rows).
// MT = 1: 2 pipeline stages and two CTAs per SM, so that one's epilogue
// overlaps the other's loads and MMAs; MT = 2 fills TMEM (512 columns): one
// CTA per SM with 3 stages.
// MNA / MNB: the operand is read MN-major from a row-major [rows][cols]
// array whose rows are the reduction index (the weight gradients dZ^T H read
// straight from the row-major dZ and H): TMA boxes of 64 columns x 64 rows,
// one per 64 output rows (A) or columns (B), 8 KB each.
template <int BN, int MT>
struct GemmShape {
  static constexpr int kStages = MT == 2 ? 3 : 2;
  static constexpr int A_BYTES = MT * BM * BK * 2, B_BYTES = BN * BK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr uint32_t TCOLS = MT * BN < 32 ? 32 : MT * BN;
  static constexpr int SMEM = kStages * STAGE + 1024 + 256;
};

template <int BN, int EPI, int MT, int MNA, int MNB>
__global__ void __launch_bounds__(192, MT == 2 ? 1 : 2)
    umma_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                     const __grid_constant__ CUtensorMap tmB, const GemmArgs p) {
  using S = GemmShape<BN, MT>;
  constexpr int kStages = S::kStages, A_BYTES = S::A_BYTES, STAGE = S::STAGE;
  constexpr uint32_t TCOLS = S::TCOLS;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * STAGE);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 1);
  int* s_ok = reinterpret_cast<int*>(slot + 1);  // the column-sum warps' shared wait outcome
  const uint32_t sbase = smem_u32(smem);
  // the epilogue warps sum A's columns from each stage while the MMAs run
  // (the weight-gradient GEMMs are bound by HBM; their epilogue warps idle)
  constexpr bool COLSUM = EPI == EPI_PARTIAL && MNA && MT == 2;
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * kStages,
                 done = full0 + 16 * kStages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kb0 = blockIdx.z * p.kb_per_split;
  const int nkb = min(p.kb_per_split, p.kb_total - kb0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, COLSUM ? 2 : 1);  // (+ the column-sum warps)
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(slot), TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  if (warp == 4) {
    // TMA producer
    if (lane == 0 && nkb > 0 && !p.inject_no_loads) {
      int issued = 0;
      for (int i = 0; i < nkb; ++i) {
        const int s = i % kStages;
        const uint32_t ph = (uint32_t)(i / kStages) & 1u;
        if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, p.status, p.wait_ns)) break;
        mbar_expect_tx(full0 + 8 * s, STAGE);
        const uint32_t sa = sbase + s * STAGE;
        if (MNA) {
#pragma unroll
          for (int j = 0; j < 2 * MT; ++j)
            tma_load_2d(sa + j * 8192, &tmA, full0 + 8 * s, m0 * MT + 64 * j, (kb0 + i) * BK);
        } else {
          tma_load_2d(sa, &tmA, full0 + 8 * s, (kb0 + i) * BK, m0 * MT);
        }
        if (MNB) {
#pragma unroll
          for (int j = 0; j < BN / 64; ++j)
            tma_load_2d(sa + A_BYTES + j * 8192, &tmB, full0 + 8 * s, n0 + 64 * j,
                        (kb0 + i) * BK);
        } else {
          tma_load_2d(sa + A_BYTES, &tmB, full0 + 8 * s, (kb0 + i) * BK, n0);
        }
        issued = i + 1;
      }
      // every load issued has landed before the CTA may exit
      for (int i = issued - kStages < 0 ? 0 : issued - kStages; i < issued; ++i)
        mbar_wait(full0 + 8 * (i % kStages), (uint32_t)(i / kStages) & 1u, p.status, p.wait_ns);
    }
  } else if (warp == 5) {
    // MMA issuer
    if (lane == 0 && nkb > 0) {
      constexpr uint32_t idesc = idesc_bf16(BM, BN, MNA, MNB);
      for (int i = 0; i < nkb; ++i) {
        const int s = i % kStages;
        const uint32_t ph = (uint32_t)(i / kStages) & 1u;
        if (!mbar_wait(full0 + 8 * s, ph, p.status, p.wait_ns)) break;
        tc_fence_after();
        const uint32_t sa = sbase + s * STAGE, sb = sa + A_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
#pragma unroll
          for (int t = 0; t < MT; ++t) {
            // K step of 16: 32 bytes along a K-major row, two 8-row groups MN-major
            const uint64_t da = MNA ? sw128_mn_desc(sa + t * 16384 + 2048 * k)
                                    : sw128_desc(sa + t * BM * 128 + 32 * k);
            const uint64_t db = MNB ? sw128_mn_desc(sb + 2048 * k) : sw128_desc(sb + 32 * k);
            umma_bf16(tmem + (uint32_t)(t * BN), da, db, idesc, (i > 0 || k > 0) ? 1u : 0u);
          }
        umma_commit(empty0 + 8 * s);
      }
      umma_commit(done);  // completes once every MMA issued above has
    }
  } else {
    float cs0 = 0.f, cs1 = 0.f;  // COLSUM: columns 2 tid, 2 tid + 1 of A
    bool cs_ok = true;
    if (COLSUM) {
      // A's 64-column chunk tid / 32, 4-byte word (tid % 32) of each 128-byte
      // row (chunk (tid % 32) / 4 of the row, under the swizzle)
      const int tid = threadIdx.x;
      const uint32_t col_off = (uint32_t)(tid >> 5) * 8192u + 4u * (uint32_t)(tid & 3);
      const uint32_t chunk = (uint32_t)((tid & 31) >> 2);
      for (int i = 0; i < nkb; ++i) {
        const int s = i % kStages;
        // one thread waits, the others follow the barrier (all take one branch)
        if (threadIdx.x == 0)
          *s_ok = mbar_wait(full0 + 8 * s, (uint32_t)(i / kStages) & 1u, p.status, p.wait_ns);
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (!(cs_ok = *s_ok != 0)) break;
        const uint8_t* st = smem + s * STAGE + col_off;
#pragma unroll 8
        for (int r = 0; r < BK; ++r) {
          const uint32_t w = *reinterpret_cast<const uint32_t*>(
              st + (r >> 3) * 1024 + (r & 7) * 128 + ((chunk ^ (uint32_t)(r & 7)) << 4));
          cs0 += __uint_as_float(w << 16);
          cs1 += __uint_as_float(w & 0xFFFF0000u);
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");  // all four warps have read stage s
        if (threadIdx.x == 0) mbar_arrive(empty0 + 8 * s);
      }
    }
    // epilogue: warp w owns TMEM lanes / output rows 32 w .. 32 w + 31
    if (nkb > 0 && cs_ok && mbar_wait(done, 0, p.status, p.wait_ns)) {
      tc_fence_after();
#pragma unroll 1
      for (int t = 0; t < MT; ++t) {
        const int m = (m0 * MT + t * BM) + warp * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * BN + c * 32), v);
          epilogue<EPI>(p, m, n0 + c * 32, v);
        }
      }
      if (COLSUM) {
        atomicAdd(p.dbias + (size_t)(2 * threadIdx.x) * p.ldb, cs0);
        atomicAdd(p.dbias + (size_t)(2 * threadIdx.x + 1) * p.ldb, cs1);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TCOLS);
  }
}

// ---- element-wise kernels ----------------------------------------------------
struct Times {
  float t[kMaxFrames];
};

// offsets in the packed parameter vector, [W_0, b_0, W_1, b_1, ..., W_head, b_head]
__host__ __device__ constexpr size_t bias_off_dev(int l) {
  return l == 0 ? (size_t)kW * kIn
                : (size_t)kW * kIn + kW + (size_t)(l - 1) * ((size_t)kW * kW + kW) + (size_t)kW * kW;
}
__host__ __device__ constexpr size_t head_bias_off_dev() {
  return (size_t)kW * kIn + kW + (size_t)(kDepth - 1) * ((size_t)kW * kW + kW) + 3 * kW;
}

// fp32 packed parameters -> bf16 W and W^T of every layer (head padded to 32 rows)
__global__ void mlp_prep_weights_kernel(const float* __restrict__ theta,
                                        __nv_bfloat16* __restrict__ wb,
                                        __nv_bfloat16* __restrict__ wt) {
  // packed offsets: layer l (0..7) W at off_w(l), then b; head after
  const int K0 = kIn;
  const size_t total = (size_t)kW * K0 + (size_t)(kDepth - 1) * kW * kW + (size_t)kHeadRows * kW;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int l, o, i;
    size_t src, dstb, dstt;
    if (e < (size_t)kW * K0) {
      l = 0;
      o = (int)(e / K0), i = (int)(e % K0);
      src = (size_t)o * K0 + i;
      dstb = e;
      dstt = (size_t)i * kW + o;
    } else if (e < (size_t)kW * K0 + (size_t)(kDepth - 1) * kW * kW) {
      const size_t r = e - (size_t)kW * K0;
      l = 1 + (int)(r / ((size_t)kW * kW));
      const size_t q = r % ((size_t)kW * kW);
      o = (int)(q / kW), i = (int)(q % kW);
      const size_t base = (size_t)kW * K0 + kW + (size_t)(l - 1) * ((size_t)kW * kW + kW);
      src = base + q;
      dstb = e;
      dstt = (size_t)kW * K0 + (size_t)(l - 1) * kW * kW + (size_t)i * kW + o;
    } else {
      const size_t r = e - (size_t)kW * K0 - (size_t)(kDepth - 1) * kW * kW;
      l = kDepth;
      o = (int)(r / kW), i = (int)(r % kW);
      const size_t base = (size_t)kW * K0 + kW + (size_t)(kDepth - 1) * ((size_t)kW * kW + kW);
      src = o < 3 ? base + (size_t)o * kW + i : 0;
      dstb = e;
      dstt = (size_t)kW * K0 + (size_t)(kDepth - 1) * kW * kW + (size_t)i * kHeadRows + o;
    }
    const float w = (l == kDepth && o >= 3) ? 0.f : theta[src];
    wb[dstb] = __float2bfloat16_rn(w);
    wt[dstt] = __float2bfloat16_rn(w);
  }
}

// positional encoding of row m = b N + g (zeros for m >= M)
__device__ __forceinline__ void encode_row(const float* __restrict__ means, const Times& tm, int N,
                                           int M, float inv_scale, int m, float* e) {
#pragma unroll
  for (int c = 0; c < kIn; ++c) e[c] = 0.f;
  if (m < M) {
    const int b = m / N, g = m - b * N;
    float x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = means[(size_t)g * 3 + a] * inv_scale;
    const float t = tm.t[b];
#pragma unroll
    for (int a = 0; a < 3; ++a) e[a] = x[a];
    float f = 1.f;
#pragma unroll
    for (int l = 0; l < kFreq; ++l, f *= 2.f) {
#pragma unroll
      for (int a = 0; a < 3; ++a) sincospif(f * x[a], &e[3 + 6 * l + a], &e[6 + 6 * l + a]);
    }
    e[63] = t;
    f = 1.f;
#pragma unroll
    for (int l = 0; l < kFreq; ++l, f *= 2.f) sincospif(f * t, &e[64 + 2 * l], &e[65 + 2 * l]);
  }
}

// positional encoding of row m = b N + g into enc[m][0..127]
__global__ void mlp_encode_kernel(const float* __restrict__ means, Times tm, int N, int B,
                                  float inv_scale, int M_pad, __nv_bfloat16* __restrict__ enc) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M_pad) return;
  float e[kIn];
  encode_row(means, tm, N, N * B, inv_scale, m, e);
#pragma unroll
  for (int q = 0; q < kIn / 32; ++q) store_row_bf16(enc + (size_t)m * kIn + 32 * q, e + 32 * q);
}

// dL/d(delta) fp32 [M][3] -> bf16 [M_pad][32] and its transpose [32][M_pad]
// (and the head's bias gradient, the column sums of the rounded values)
__global__ void __launch_bounds__(128)
    mlp_head_grad_kernel(const float* __restrict__ dd, int M, int M_pad,
                         __nv_bfloat16* __restrict__ dz, __nv_bfloat16* __restrict__ dzt,
                         float* __restrict__ dbias, int ldb) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  float v[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = 0.f;
  if (m < M) {
#pragma unroll
    for (int j = 0; j < 3; ++j) v[j] = dd[(size_t)m * 3 + j];
  }
  if (m < M_pad) {
    store_row_bf16(dz + (size_t)m * kHeadRows, v);
#pragma unroll
    for (int j = 0; j < kHeadRows; ++j) dzt[(size_t)j * M_pad + m] = __float2bfloat16_rn(v[j]);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float b = __bfloat162float(__float2bfloat16_rn(v[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if ((threadIdx.x & 31) == 0 && b != 0.f) atomicAdd(dbias + (size_t)j * ldb, b);
  }
}

// dL/d(means) from the encoding's gradient (the position part, columns
// 0..62), summed over the frames: one warp per Gaussian.  The frames' rows
// are summed first (coalesced, lanes over columns), then each lane applies
// the derivative of its columns' encoding -- d sin(f pi x)/dx = f pi cos(f pi x),
// d cos(f pi x)/dx = -f pi sin(f pi x) -- and the warp reduces per axis.
__global__ void __launch_bounds__(256)
    mlp_encode_bwd_kernel(const float* __restrict__ means, const float* __restrict__ denc, int N,
                          int B, float inv_scale, float* __restrict__ dmeans) {
  const int g = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (g >= N) return;
  float d0 = 0.f, d1 = 0.f;  // columns lane and lane + 32, summed over the frames
  for (int b = 0; b < B; ++b) {
    const float* row = denc + ((size_t)b * N + g) * kIn;
    d0 += __ldg(row + lane);
    if (lane < 31) d1 += __ldg(row + 32 + lane);
  }
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = lane + 32 * h;
    const float d = h ? d1 : d0;
    if (c < 3) {
      acc[c] += d;
    } else if (c < 63) {
      const int l = (c - 3) / 6, w = (c - 3) - 6 * l, a = w < 3 ? w : w - 3;
      const float f = (float)(1 << l);
      const float x = __ldg(means + (size_t)g * 3 + a) * inv_scale;
      float sn, cs;
      sincospif(f * x, &sn, &cs);
      const float term = f * 3.14159265358979323846f * (w < 3 ? cs * d : -sn * d);
      acc[0] += a == 0 ? term : 0.f;
      acc[1] += a == 1 ? term : 0.f;
      acc[2] += a == 2 ? term : 0.f;
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], off);
  if (lane == 0)
    for (int a = 0; a < 3; ++a) dmeans[(size_t)g * 3 + a] = acc[a] * inv_scale;
}

// extended weight gradients [rows][K + ext] -> packed d_theta (W then b)
__global__ void mlp_unpack_grads_kernel(const float* __restrict__ dwx, float* __restrict__ dth) {
  const size_t total = (size_t)kW * (kIn + 1) + (size_t)(kDepth - 1) * kW * (kW + 1) + 3 * (kW + 1);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    // locate layer
    size_t r = e, src_base = 0;
    int K = kIn, rows = kW, l = 0;
    for (;;) {
      const size_t n = (size_t)rows * (K + 1);
      if (r < n) break;
      r -= n;
      src_base += (size_t)(l == kDepth ? kHeadRows : kW) * (K + kExt);
      ++l;
      K = kW;
      rows = l == kDepth ? 3 : kW;
    }
    const int ld = K + kExt;
    float v;
    if (r < (size_t)rows * K) {
      const int o = (int)(r / K), i = (int)(r % K);
      v = dwx[src_base + (size_t)o * ld + i];
    } else {
      const int o = (int)(r - (size_t)rows * K);
      v = dwx[src_base + (size_t)o * ld + K];
    }
    dth[e] = v;
  }
}

// sum of the row-split partials [splits][256][K] -> dW block [256][ld]
__global__ void mlp_reduce_dw_kernel(const float* __restrict__ part, int splits, int K,
                                     float* __restrict__ dw, int ld) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kW * K) return;
  const size_t stride = (size_t)kW * K;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += part[(size_t)z * stride + e];
  const int o = e / K, i = e - o * K;
  dw[(size_t)o * ld + i] = s;
}

// ---- fused forward (inference): all layers of 128-row tiles in one CTA -------
// The activations never leave shared memory: the epilogue warps write each
// layer's output (bias, ReLU, BF16) straight into the 128 x 256 operand tile
// of the next layer, in the swizzled K-major layout of the MMA descriptors,
// while a TMA warp streams the layers' weights through a 3-stage ring.  A CTA
// works on two tiles at once (two activation tiles, two TMEM accumulators),
// alternating (layer, tile) items so that the epilogue of one tile runs while
// the tensor core computes the other.  The arithmetic and its order are those
// of the layer-by-layer forward, so the outputs agree bit for bit; nothing is
// kept for a backward.
constexpr int kFusedStages = 3;
constexpr int kPair = 2;                   // tiles in flight per CTA
constexpr int kActBytes = BM * kW * 2;     // 64 KB per tile
constexpr int kWStageBytes = kW * BK * 2;  // 32 KB (a 256-row k-block of W)
constexpr int kFusedSmem = kPair * kActBytes + kFusedStages * kWStageBytes + 1024 + 256;

struct FusedMaps {
  CUtensorMap w[kDepth + 1];  // bf16 W of the hidden layers (256 rows), head (32 rows)
  CUtensorMap enc;            // training forward: the encoding [Mp][128] (stores)
  CUtensorMap act;            // H (forward) or dZ (backward) of all layers [8 Mp][256] (stores)
};

// byte offset of element (r, c) of an activation tile: 64-column blocks of
// 16 KB, rows 128 bytes apart in 1024-byte 8-row atoms, 16-byte chunk j of
// row r at chunk j ^ (r & 7) (the 128-byte swizzle)
__device__ __forceinline__ uint32_t act_off(int r, int c) {
  const int kb = c >> 6, cc = c & 63;
  return (uint32_t)(kb * 16384 + (r >> 3) * 1024 + (r & 7) * 128 +
                    ((((cc >> 3) ^ (r & 7)) << 4) | ((cc & 7) << 1)));
}
__device__ __forceinline__ void store_act32(uint8_t* act, int r, int c, const float* v) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint4 u;
    uint32_t* w = reinterpret_cast<uint32_t*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __nv_bfloat162 h = __floats2bfloat162_rn(v[8 * q + 2 * i], v[8 * q + 2 * i + 1]);
      w[i] = *reinterpret_cast<uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(act + act_off(r, c + 8 * q)) = u;
  }
}

// the same with the ReLU folded into the conversion: each BF16 value is
// bf16_rn(v) clamped at zero, which equals bf16_rn(max(v, 0))
__device__ __forceinline__ void store_act32_relu(uint8_t* act, int r, int c, const float* v) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint4 u;
    uint32_t* w = reinterpret_cast<uint32_t*>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;"
          : "=r"(w[i])
          : "f"(v[8 * q + 2 * i + 1]), "f"(v[8 * q + 2 * i]));
    *reinterpret_cast<uint4*>(act + act_off(r, c + 8 * q)) = u;
  }
}

// warps 0-7: epilogue (warp w: TMEM lanes / rows 32 (w % 4) .. + 31, columns
// 128 (w / 4) .. + 127); warp 8: TMA; warp 9: MMA
constexpr int kFusedEpiWarps = 8;
constexpr int kFusedThreads = 32 * (kFusedEpiWarps + 2);

// What a training forward keeps for the backward (TRAIN): the encoded input
// and every hidden activation (row-major BF16, stored by TMA from the tile in
// shared memory through maps.enc / maps.act), and the ReLU masks as bits
// ([layer][Mp][8] words) -- the same values the layer-by-layer forward
// stores.  The stores of tile t are issued (and waited for before the tile is
// written again) by epilogue thread 32 t.
struct FusedKeep {
  uint32_t* bits;
  int Mp;
};

template <bool TRAIN>
__global__ void __launch_bounds__(kFusedThreads, 1)
    mlp_fused_fwd_kernel(const __grid_constant__ FusedMaps maps, const float* __restrict__ theta,
                         const float* __restrict__ means, Times tm, int N, int M, int n_tiles,
                         float inv_scale, float* __restrict__ delta, int* status,
                         unsigned long long wait_ns, int inject_no_loads, FusedKeep keep) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(smem + kPair * kActBytes + kFusedStages * kWStageBytes);
  // bars: full[S], empty[S], acc_ready[kPair], act_ready[kPair]
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2 * kFusedStages + 2 * kPair);
  int* s_ok = reinterpret_cast<int*>(slot + 1);  // the epilogue's shared wait outcome
  const uint32_t act_s = smem_u32(smem), w_s = act_s + kPair * kActBytes;
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * kFusedStages;
  const uint32_t acc0 = full0 + 16 * kFusedStages, actr0 = acc0 + 8 * kPair;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_pairs = (n_tiles + kPair - 1) / kPair;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kFusedStages; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    for (int t = 0; t < kPair; ++t) {
      mbar_init(acc0 + 8 * t, 1);
      mbar_init(actr0 + 8 * t, 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(slot), (uint32_t)(kPair * kW));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  if (warp == kFusedEpiWarps) {
    // weights of every (layer, tile) item, k-block by k-block
    if (lane == 0 && !inject_no_loads) {
      int it = 0;
      bool ok = true;
      for (int pr = blockIdx.x; ok && pr < n_pairs; pr += gridDim.x)
        for (int l = 0; ok && l <= kDepth; ++l)
          for (int t = 0; ok && t < kPair; ++t) {
            const int nkb = (l == 0 ? kIn : kW) / BK;
            const uint32_t bytes = (uint32_t)(l == kDepth ? kHeadRows : kW) * BK * 2;
            for (int kb = 0; kb < nkb; ++kb, ++it) {
              const int s = it % kFusedStages;
              if (!(ok = mbar_wait(empty0 + 8 * s, ((uint32_t)(it / kFusedStages) & 1u) ^ 1u,
                                   status, wait_ns)))
                break;
              mbar_expect_tx(full0 + 8 * s, bytes);
              tma_load_2d(w_s + s * kWStageBytes, &maps.w[l], full0 + 8 * s, kb * BK, 0);
            }
          }
      // every load issued has landed before the CTA may exit
      for (int i = it - kFusedStages < 0 ? 0 : it - kFusedStages; i < it; ++i)
        mbar_wait(full0 + 8 * (i % kFusedStages), (uint32_t)(i / kFusedStages) & 1u, status,
                  wait_ns);
    }
  } else if (warp == kFusedEpiWarps + 1) {
    if (lane == 0) {
      int it = 0;
      uint32_t act_ph[kPair] = {0, 0};
      bool ok = true;
      for (int pr = blockIdx.x; ok && pr < n_pairs; pr += gridDim.x)
        for (int l = 0; ok && l <= kDepth; ++l)
          for (int t = 0; ok && t < kPair; ++t) {
            if (!(ok = mbar_wait(actr0 + 8 * t, act_ph[t], status, wait_ns))) break;
            act_ph[t] ^= 1u;
            tc_fence_after();
            const int nkb = (l == 0 ? kIn : kW) / BK;
            const uint32_t idesc = l == kDepth ? idesc_bf16(BM, kHeadRows) : idesc_bf16(BM, kW);
            const uint32_t d = tmem + (uint32_t)(t * kW);
            for (int kb = 0; kb < nkb; ++kb, ++it) {
              const int s = it % kFusedStages;
              if (!(ok = mbar_wait(full0 + 8 * s, (uint32_t)(it / kFusedStages) & 1u, status,
                                   wait_ns)))
                break;
              tc_fence_after();
              const uint32_t sa = act_s + t * kActBytes + kb * 16384, sb = w_s + s * kWStageBytes;
#pragma unroll
              for (int k = 0; k < BK / 16; ++k)
                umma_bf16(d, sw128_desc(sa + 32 * k), sw128_desc(sb + 32 * k), idesc,
                          (kb > 0 || k > 0) ? 1u : 0u);
              umma_commit(empty0 + 8 * s);
            }
            umma_commit(acc0 + 8 * t);
          }
    }
  } else {
    // epilogue warps: row r of every tile, one half of the columns
    const int q = warp & 3, half = warp >> 2;
    const int r = q * 32 + lane;
    uint32_t acc_ph[kPair] = {0, 0};
    bool ok = true;
    for (int pr = blockIdx.x; ok && pr < n_pairs; pr += gridDim.x) {
      for (int t = 0; t < kPair; ++t) {
        if (half == 0) {
          float e[kIn];
          const int m = (pr * kPair + t) * BM + r;
          encode_row(means, tm, N, M, inv_scale, m, e);
          uint8_t* act = smem + t * kActBytes;
#pragma unroll
          for (int c = 0; c < kIn; c += 32) store_act32(act, r, c, e + c);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (threadIdx.x == 0) mbar_arrive(actr0 + 8 * t);
        if (TRAIN && threadIdx.x == 32 * t && pr * kPair + t < n_tiles) {
          for (int kb = 0; kb < kIn / BK; ++kb)
            tma_store_2d(&maps.enc, act_s + t * kActBytes + kb * 16384, kb * BK,
                         (pr * kPair + t) * BM);
          bulk_commit();
        }
      }
      for (int l = 0; ok && l <= kDepth; ++l)
        for (int t = 0; t < kPair; ++t) {
          // one thread waits, the other epilogue threads follow the barrier, so
          // that all 128 take the same branch (no split at the named barriers)
          if (threadIdx.x == 0)
            *s_ok = mbar_wait(acc0 + 8 * t, acc_ph[t], status, wait_ns) ? 1 : 0;
          // the tile's last store has read it before it is written again
          if (TRAIN && threadIdx.x == 32 * t) bulk_wait_read();
          asm volatile("bar.sync 1, 256;" ::: "memory");
          // (every step ends at a named barrier that all epilogue threads reach
          // after reading the flag, so thread 0 rewrites it only afterwards)
          if (!(ok = *s_ok != 0)) break;
          acc_ph[t] ^= 1u;
          tc_fence_after();
          const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * kW);
          uint8_t* act = smem + t * kActBytes;
          if (l < kDepth) {
            const float* bias = theta + bias_off_dev(l);
#pragma unroll 1
            for (int c0 = half * (kW / 2); c0 < (half + 1) * (kW / 2); c0 += 64) {
              float vv[64];
              tmem_ld64(trow + (uint32_t)c0, vv);
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                float* v = vv + 32 * h;
                const int c = c0 + 32 * h;
                const float4* b4 = reinterpret_cast<const float4*>(bias + c);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const float4 b = __ldg(b4 + j);
                  v[4 * j] += b.x;
                  v[4 * j + 1] += b.y;
                  v[4 * j + 2] += b.z;
                  v[4 * j + 3] += b.w;
                }
                store_act32_relu(act, r, c, v);  // (the mask bits below: v > 2^-134
                                                 // before or after the ReLU alike)
                const int m = (pr * kPair + t) * BM + r;
                if (TRAIN && m < keep.Mp)
                  keep.bits[((size_t)l * keep.Mp + m) * (kW / 32) + c / 32] = relu_bits(v);
              }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (threadIdx.x == 0) mbar_arrive(actr0 + 8 * t);
            if (TRAIN && threadIdx.x == 32 * t && pr * kPair + t < n_tiles) {
              for (int kb = 0; kb < kW / BK; ++kb)
                tma_store_2d(&maps.act, act_s + t * kActBytes + kb * 16384, kb * BK,
                             l * keep.Mp + (pr * kPair + t) * BM);
              bulk_commit();
            }
          } else {
            if (half == 0) {
              float v[32];
              tmem_ld32(trow, v);
              const float* bias = theta + head_bias_off_dev();
              const int m = (pr * kPair + t) * BM + r;
              if (m < M)
                for (int j = 0; j < 3; ++j) delta[(size_t)m * 3 + j] = v[j] + __ldg(bias + j);
            }
            tc_fence_before();
            asm volatile("bar.sync 1, 256;" ::: "memory");  // TMEM drained before the next pair
          }
        }
    }
    if (TRAIN && (threadIdx.x & 31) == 0) bulk_wait_all();  // the stores are done
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)(kPair * kW));
  }
}

// ---- fused backward: the dZ chain of 128-row tiles kept in shared memory ----
// Step s = 0 forms dZ_7 = (dZ_head W_head) * mask_7 from dL/d(delta); steps
// s = 1..7 form dZ_{7-s} = (dZ_{8-s} W_{8-s}) * mask_{7-s}; step 8 forms the
// encoding's gradient dZ_0 W_0 (FP32).  Each dZ tile goes to shared memory as
// the next step's operand and from there by TMA (maps.act, row-major) to
// global memory for the weight gradients (whose GEMMs also form the bias
// gradients, the column sums).  The same operands and order as the
// one-GEMM-per-layer backward: bit-identical dZ.
constexpr int kBwdStages = kFusedStages;
constexpr int kBwdSmem = kFusedSmem;

struct FusedBwdArgs {
  const float* dd;      // dL/d(delta) [M][3]
  const uint32_t* bits; // ReLU masks [layer][Mp][8]
  float* denc;          // [Mp][128] (out)
  int M, Mp, n_tiles;
};

__global__ void __launch_bounds__(kFusedThreads, 1)
    mlp_fused_bwd_kernel(const __grid_constant__ FusedMaps maps, const FusedBwdArgs a,
                         int* status, unsigned long long wait_ns, int inject_no_loads) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(smem + kPair * kActBytes + kBwdStages * kWStageBytes);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2 * kBwdStages + 2 * kPair);
  int* s_ok = reinterpret_cast<int*>(slot + 1);
  const uint32_t act_s = smem_u32(smem), w_s = act_s + kPair * kActBytes;
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * kBwdStages;
  const uint32_t acc0 = full0 + 16 * kBwdStages, actr0 = acc0 + 8 * kPair;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_pairs = (a.n_tiles + kPair - 1) / kPair;
  constexpr int kSteps = kDepth + 1;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kBwdStages; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    for (int t = 0; t < kPair; ++t) {
      mbar_init(acc0 + 8 * t, 1);
      mbar_init(actr0 + 8 * t, 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(slot), (uint32_t)(kPair * kW));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  if (warp == kFusedEpiWarps) {
    // W^T of the head (step 0) and of layers 7..0 (steps 1..8)
    if (lane == 0 && !inject_no_loads) {
      int it = 0;
      bool ok = true;
      for (int pr = blockIdx.x; ok && pr < n_pairs; pr += gridDim.x)
        for (int st = 0; ok && st < kSteps; ++st)
          for (int t = 0; ok && t < kPair; ++t) {
            const int nkb = st == 0 ? 1 : kW / BK;
            for (int kb = 0; kb < nkb; ++kb, ++it) {
              const int s = it % kBwdStages;
              if (!(ok = mbar_wait(empty0 + 8 * s, ((uint32_t)(it / kBwdStages) & 1u) ^ 1u,
                                   status, wait_ns)))
                break;
              mbar_expect_tx(full0 + 8 * s, (uint32_t)kWStageBytes);
              tma_load_2d(w_s + s * kWStageBytes, &maps.w[st == 0 ? kDepth : kDepth - st],
                          full0 + 8 * s, kb * BK, 0);
            }
          }
      for (int i = it - kBwdStages < 0 ? 0 : it - kBwdStages; i < it; ++i)
        mbar_wait(full0 + 8 * (i % kBwdStages), (uint32_t)(i / kBwdStages) & 1u, status,
                  wait_ns);
    }
  } else if (warp == kFusedEpiWarps + 1) {
    if (lane == 0) {
      int it = 0;
      uint32_t act_ph[kPair] = {0, 0};
      bool ok = true;
      constexpr uint32_t idesc = idesc_bf16(BM, kW);
      for (int pr = blockIdx.x; ok && pr < n_pairs; pr += gridDim.x)
        for (int st = 0; ok && st < kSteps; ++st)
          for (int t = 0; ok && t < kPair; ++t) {
            if (!(ok = mbar_wait(actr0 + 8 * t, act_ph[t], status, wait_ns))) break;
            act_ph[t] ^= 1u;
            tc_fence_after();
            const int nkb = st == 0 ? 1 : kW / BK;
            const uint32_t d = tmem + (uint32_t)(t * kW);
            for (int kb = 0; kb < nkb; ++kb, ++it) {
              const int s = it % kBwdStages;
              if (!(ok = mbar_wait(full0 + 8 * s, (uint32_t)(it / kBwdStages) & 1u, status,
                                   wait_ns)))
                break;
              tc_fence_after();
              const uint32_t sa = act_s + t * kActBytes + kb * 16384, sb = w_s + s * kWStageBytes;
#pragma unroll
              for (int k = 0; k < BK / 16; ++k)
                umma_bf16(d, sw128_desc(sa + 32 * k), sw128_desc(sb + 32 * k), idesc,
                          (kb > 0 || k > 0) ? 1u : 0u);
              umma_commit(empty0 + 8 * s);
            }
            umma_commit(acc0 + 8 * t);
          }
    }
  } else {
    const int q = warp & 3, half = warp >> 2;
    const int r = q * 32 + lane;
    uint32_t acc_ph[kPair] = {0, 0};
    // the ReLU mask words of this thread's row and column half, one step
    // ahead: a tile's next layer is loaded while this one is processed
    uint4 nb[kPair];
    auto load_bits = [&](int layer, int m) {
      return m < a.Mp ? __ldg(reinterpret_cast<const uint4*>(
                                  a.bits + ((size_t)layer * a.Mp + m) * (kW / 32)) +
                              half)
                      : make_uint4(0u, 0u, 0u, 0u);
    };
    bool ok = true;
    for (int pr = blockIdx.x; ok && pr < n_pairs; pr += gridDim.x) {
#pragma unroll
      for (int t = 0; t < kPair; ++t) {
        // step 0's operand: BF16 dL/d(delta) in columns 0..2 of k-block 0
        const int m = (pr * kPair + t) * BM + r;
        nb[t] = load_bits(kDepth - 1, m);
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0.f;
        if (half == 0 && m < a.M)
          for (int j = 0; j < 3; ++j) v[j] = a.dd[(size_t)m * 3 + j];
        store_act32(smem + t * kActBytes, r, 32 * half, v);  // (free: waited at step 8)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (threadIdx.x == 0) mbar_arrive(actr0 + 8 * t);
      }
      for (int st = 0; ok && st < kSteps; ++st)
#pragma unroll
        for (int t = 0; t < kPair; ++t) {
          if (threadIdx.x == 0)
            *s_ok = mbar_wait(acc0 + 8 * t, acc_ph[t], status, wait_ns) ? 1 : 0;
          // the tile's last store has read it before it is written again
          if (threadIdx.x == 32 * t) bulk_wait_read();
          asm volatile("bar.sync 1, 256;" ::: "memory");
          if (!(ok = *s_ok != 0)) break;  // (rewritten only after the step's last barrier)
          acc_ph[t] ^= 1u;
          tc_fence_after();
          const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * kW);
          const int m = (pr * kPair + t) * BM + r;
          if (st < kDepth) {
            const int j = kDepth - 1 - st;  // the layer whose dZ this step forms
            uint8_t* act = smem + t * kActBytes;
            const uint4 mk = nb[t];
            if (j > 0) nb[t] = load_bits(j - 1, m);
#pragma unroll 1
            for (int h2 = 0; h2 < 2; ++h2) {
              const int c0 = half * (kW / 2) + 64 * h2;
              const uint32_t mk0 = h2 ? mk.z : mk.x, mk1 = h2 ? mk.w : mk.y;
              float vv[64];
              tmem_ld64(trow + (uint32_t)c0, vv);
#pragma unroll
              for (int k = 0; k < 32; ++k) {
                if (!((mk0 >> k) & 1u)) vv[k] = 0.f;
                if (!((mk1 >> k) & 1u)) vv[32 + k] = 0.f;
              }
              store_act32(act, r, c0, vv);
              store_act32(act, r, c0 + 32, vv + 32);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (threadIdx.x == 0) mbar_arrive(actr0 + 8 * t);
            if (threadIdx.x == 32 * t && pr * kPair + t < a.n_tiles) {
              for (int kb = 0; kb < kW / BK; ++kb)
                tma_store_2d(&maps.act, act_s + t * kActBytes + kb * 16384, kb * BK,
                             j * a.Mp + (pr * kPair + t) * BM);
              bulk_commit();
            }
          } else {
            if (half == 0) {
#pragma unroll 1
              for (int c = 0; c < kIn; c += 32) {
                float v[32];
                tmem_ld32(trow + (uint32_t)c, v);
                if (m < a.Mp) {
                  float4* d = reinterpret_cast<float4*>(a.denc + (size_t)m * kIn + c);
#pragma unroll
                  for (int k = 0; k < 8; ++k)
                    d[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                }
              }
            }
            tc_fence_before();
            asm volatile("bar.sync 1, 256;" ::: "memory");  // TMEM drained before the next pair
          }
        }
    }
    if ((threadIdx.x & 31) == 0) bulk_wait_all();  // the stores are done
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)(kPair * kW));
  }
}

// ---- host side -----------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// bf16 matrix [rows][cols] with row stride ld elements; boxes of 64 columns x
// box_rows with the 128-byte swizzle
bool make_map(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
              uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * 2) % 16 != 0) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int EPI, int MT = 1, int MNA = 0, int MNB = 0>
bool gemm(const CUtensorMap& a, const CUtensorMap& b, const GemmArgs& args, int m_tiles,
          int n_tiles, int splits, cudaStream_t st) {
  constexpr int smem = GemmShape<BN, MT>::SMEM;
  static PerDeviceOnce configured;
  if (!configured.run([] {
        return cudaFuncSetAttribute(umma_gemm_kernel<BN, EPI, MT, MNA, MNB>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    smem) == cudaSuccess;
      }))
    return false;
  umma_gemm_kernel<BN, EPI, MT, MNA, MNB>
      <<<dim3(m_tiles, n_tiles, splits), 192, smem, st>>>(a, b, args);
  count_launches(1);
  return true;
}

struct MlpLayout {
  int N, B, M, M_pad;
  size_t off_status, off_wb, off_wt, off_enc, off_h, off_bits, off_dz, off_dzh, off_dzht,
      off_denc, off_dwx, off_part, total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t dwx_floats() {
  return (size_t)kW * (kIn + kExt) + (size_t)(kDepth - 1) * kW * (kW + kExt) +
         (size_t)kHeadRows * (kW + kExt);
}
size_t wb_elems() {
  return (size_t)kW * kIn + (size_t)(kDepth - 1) * kW * kW + (size_t)kHeadRows * kW;
}

MlpLayout mlp_layout(int N, int B) {
  MlpLayout L;
  memset(&L, 0, sizeof(L));
  L.N = N, L.B = B, L.M = N * B;
  L.M_pad = (L.M + BM - 1) / BM * BM;
  if (L.M_pad == 0) L.M_pad = BM;
  const size_t Mp = (size_t)L.M_pad;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at_ = o;
    o = align256(o + bytes);
    return at_;
  };
  L.off_status = take(256);
  L.off_wb = take(wb_elems() * 2);
  L.off_wt = take(wb_elems() * 2);
  L.off_enc = take(Mp * kIn * 2);                   // [Mp][128]
  L.off_h = take((size_t)kDepth * Mp * kW * 2);     // [layer][Mp][256]
  L.off_bits = take((size_t)kDepth * Mp * (kW / 32) * 4);
  L.off_dz = take((size_t)kDepth * Mp * kW * 2);    // [layer][Mp][256]
  L.off_dzh = take(Mp * kHeadRows * 2);
  L.off_dzht = take((size_t)kHeadRows * Mp * 2);
  L.off_denc = take(Mp * kIn * 4);
  L.off_dwx = take(dwx_floats() * 4);
  L.off_part = take((size_t)kMaxSplits * kW * kW * 4);
  L.total = o;
  return L;
}

// rows: below 2^27 (the stores address layer l's rows at l Mp + m with
// 32-bit TMA coordinates)
bool mlp_args_ok(int N, int B) {
  return N >= 0 && B >= 1 && B <= kMaxFrames && (int64_t)N * B < (int64_t)1 << 27;
}

// test hooks (gftorf_mlp_debug_inject): 1 = the GEMMs' load warps issue
// nothing, so the MMA and epilogue waits run out; 2 = the training forward
// and the backward's dZ chain run layer by layer (one GEMM per layer)
// instead of fused
std::atomic<int> g_inject{0};

bool fused_configured() {
  static PerDeviceOnce once;
  return once.run([] {
    return cudaFuncSetAttribute(mlp_fused_fwd_kernel<false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem) ==
               cudaSuccess &&
           cudaFuncSetAttribute(mlp_fused_fwd_kernel<true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedSmem) ==
               cudaSuccess &&
           cudaFuncSetAttribute(mlp_fused_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kBwdSmem) == cudaSuccess;
  });
}

template <typename T>
T* ptr(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<unsigned char*>(ws) + off);
}

// bf16 weights of layer l (l = kDepth: head) and their transposes
size_t wb_off(int l) {
  return l == 0 ? 0 : (size_t)kW * kIn + (size_t)(l - 1) * kW * kW;
}
size_t bias_off(int l) {  // in the packed fp32 vector
  if (l == 0) return (size_t)kW * kIn;
  return (size_t)kW * kIn + kW + (size_t)(l - 1) * ((size_t)kW * kW + kW) + (size_t)kW * kW;
}
size_t head_bias_off() {
  return (size_t)kW * kIn + kW + (size_t)(kDepth - 1) * ((size_t)kW * kW + kW) + 3 * kW;
}
size_t dwx_off(int l) {  // floats
  if (l == 0) return 0;
  return (size_t)kW * (kIn + kExt) + (size_t)(l - 1) * kW * (kW + kExt);
}

}  // namespace
}  // namespace gftorf

using namespace gftorf;

extern "C" size_t gftorf_mlp_infer_workspace_size(void) {
  return 256 + align256(2 * wb_elems() * 2);  // status word, BF16 weights and transposes
}

extern "C" size_t gftorf_mlp_workspace_size(int32_t n_gaussians, int32_t n_frames) {
  if (!mlp_args_ok(n_gaussians, n_frames)) return 0;
  return mlp_layout(n_gaussians, n_frames).total;
}

extern "C" size_t gftorf_mlp_param_count(void) {
  return (size_t)kW * kIn + kW + (size_t)(kDepth - 1) * ((size_t)kW * kW + kW) + 3 * kW + 3;
}

extern "C" gftorf_status gftorf_mlp_forward(int32_t n_gaussians, int32_t n_frames,
                                            const float* theta, const float* means,
                                            const float* times, float inv_scale, float* delta,
                                            void* workspace, size_t workspace_bytes,
                                            void* stream) {
  gftorf::TraceRange trace_("gftorf_mlp_forward");
  if (!mlp_args_ok(n_gaussians, n_frames) || !theta || !times ||
      (n_gaussians > 0 && (!means || !delta)) || !(inv_scale > 0.f))
    return GFTORF_ERR_ARG;
  const MlpLayout L = mlp_layout(n_gaussians, n_frames);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 ||
      workspace_bytes < L.total)
    return GFTORF_ERR_WORKSPACE;
  for (int b = 0; b < n_frames; ++b)
    if (!std::isfinite(times[b])) return GFTORF_ERR_ARG;
  if (!encode_fn()) return GFTORF_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* ws = workspace;
  const int Mp = L.M_pad;
  int* status = ptr<int>(ws, L.off_status);
  cudaMemsetAsync(status, 0, 256, st);  // the status word of this forward and its backward
  if (L.M == 0) return cudaGetLastError() == cudaSuccess ? GFTORF_OK : GFTORF_ERR_CUDA;
  auto* wb = ptr<__nv_bfloat16>(ws, L.off_wb);
  auto* wt = ptr<__nv_bfloat16>(ws, L.off_wt);
  mlp_prep_weights_kernel<<<4 * 152, 256, 0, st>>>(theta, wb, wt);
  Times tm;
  memset(&tm, 0, sizeof(tm));
  for (int b = 0; b < n_frames; ++b) tm.t[b] = times[b];
  auto* enc = ptr<__nv_bfloat16>(ws, L.off_enc);
  auto* H = ptr<__nv_bfloat16>(ws, L.off_h);
  const int mt = Mp / BM;
  if (g_inject.load() != 2) {
    // fused: all layers per pair of 128-row tiles, keeping the encoding, the
    // activations and the ReLU masks for the backward
    if (!fused_configured()) return GFTORF_ERR_CUDA;
    FusedMaps maps;
    for (int l = 0; l <= kDepth; ++l) {
      const int K = l == 0 ? kIn : kW, rows = l == kDepth ? kHeadRows : kW;
      if (!make_map(&maps.w[l], wb + wb_off(l), rows, K, K, rows)) return GFTORF_ERR_CUDA;
    }
    if (!make_map(&maps.enc, enc, Mp, kIn, kIn, BM) ||
        !make_map(&maps.act, H, (uint64_t)kDepth * Mp, kW, kW, BM))
      return GFTORF_ERR_CUDA;
    FusedKeep keep;
    keep.bits = ptr<uint32_t>(ws, L.off_bits), keep.Mp = Mp;
    const int sms = sm_count();
    const int n_pairs = (mt + kPair - 1) / kPair;
    const int inj = g_inject.load();
    mlp_fused_fwd_kernel<true><<<n_pairs < sms ? n_pairs : sms, kFusedThreads, kFusedSmem, st>>>(
        maps, theta, means, tm, n_gaussians, L.M, mt, inv_scale, delta, status,
        inj == 1 ? 50000000ull : 2000000000ull, inj == 1, keep);
    count_launches(2);
    return cudaGetLastError() == cudaSuccess ? GFTORF_OK : GFTORF_ERR_CUDA;
  }
  mlp_encode_kernel<<<(Mp + 127) / 128, 128, 0, st>>>(means, tm, n_gaussians, n_frames,
                                                      inv_scale, Mp, enc);
  count_launches(2);
  for (int l = 0; l < kDepth; ++l) {
    const int K = l == 0 ? kIn : kW;
    const __nv_bfloat16* in = l == 0 ? enc : H + (size_t)(l - 1) * Mp * kW;
    CUtensorMap ma, mb;
    if (!make_map(&ma, in, Mp, K, K, BM) || !make_map(&mb, wb + wb_off(l), kW, K, K, 256))
      return GFTORF_ERR_CUDA;
    GemmArgs a;
    memset(&a, 0, sizeof(a));
    a.kb_total = K / BK, a.kb_per_split = K / BK;
    a.rows_valid = Mp, a.cols_valid = kW;
    a.bias = theta + bias_off(l);
    a.out_b = H + (size_t)l * Mp * kW, a.ldo = kW;
    a.mbits = ptr<uint32_t>(ws, L.off_bits) + (size_t)l * Mp * (kW / 32);
    a.status = status;
    a.inject_no_loads = g_inject.load(std::memory_order_relaxed) == 1;
    a.wait_ns = a.inject_no_loads ? 50000000ull : 2000000000ull;
    if (!gemm<256, EPI_HIDDEN>(ma, mb, a, mt, 1, 1, st)) return GFTORF_ERR_CUDA;
  }
  {
    CUtensorMap ma, mb;
    if (!make_map(&ma, H + (size_t)(kDepth - 1) * Mp * kW, Mp, kW, kW, BM) ||
        !make_map(&mb, wb + wb_off(kDepth), kHeadRows, kW, kW, kHeadRows))
      return GFTORF_ERR_CUDA;
    GemmArgs a;
    memset(&a, 0, sizeof(a));
    a.kb_total = kW / BK, a.kb_per_split = kW / BK;
    a.rows_valid = L.M, a.cols_valid = 3;
    a.bias = theta + head_bias_off();
    a.out_f = delta;
    a.status = status;
    a.inject_no_loads = g_inject.load(std::memory_order_relaxed) == 1;
    a.wait_ns = a.inject_no_loads ? 50000000ull : 2000000000ull;
    if (!gemm<32, EPI_HEAD>(ma, mb, a, mt, 1, 1, st)) return GFTORF_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? GFTORF_OK : GFTORF_ERR_CUDA;
}

extern "C" gftorf_status gftorf_mlp_backward(int32_t n_gaussians, int32_t n_frames,
                                             const float* theta, const float* means,
                                             const float* times, float inv_scale,
                                             const float* d_delta, float* d_theta,
                                             float* d_means, void* workspace,
                                             size_t workspace_bytes, void* stream) {
  gftorf::TraceRange trace_("gftorf_mlp_backward");
  if (!mlp_args_ok(n_gaussians, n_frames) || !theta || !times || !d_theta ||
      (n_gaussians > 0 && (!means || !d_means || !d_delta)) || !(inv_scale > 0.f))
    return GFTORF_ERR_ARG;
  const MlpLayout L = mlp_layout(n_gaussians, n_frames);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 ||
      workspace_bytes < L.total)
    return GFTORF_ERR_WORKSPACE;
  if (!encode_fn()) return GFTORF_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* ws = workspace;
  const int Mp = L.M_pad;
  int* status = ptr<int>(ws, L.off_status);
  float* dwx = ptr<float>(ws, L.off_dwx);
  cudaMemsetAsync(dwx, 0, dwx_floats() * 4, st);
  if (L.M == 0) {
    mlp_unpack_grads_kernel<<<4 * 152, 256, 0, st>>>(dwx, d_theta);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? GFTORF_OK : GFTORF_ERR_CUDA;
  }
  auto* wt = ptr<__nv_bfloat16>(ws, L.off_wt);
  auto* enc = ptr<__nv_bfloat16>(ws, L.off_enc);
  auto H = [&](int l) { return ptr<__nv_bfloat16>(ws, L.off_h) + (size_t)l * Mp * kW; };
  auto* bits = ptr<uint32_t>(ws, L.off_bits);
  auto* dzh = ptr<__nv_bfloat16>(ws, L.off_dzh);
  auto* dzht = ptr<__nv_bfloat16>(ws, L.off_dzht);
  auto dz = [&](int l) { return ptr<__nv_bfloat16>(ws, L.off_dz) + (size_t)l * Mp * kW; };
  float* denc = ptr<float>(ws, L.off_denc);
  const int mt = Mp / BM;
  const int kb_rows = Mp / BK;      // k-blocks of a reduction over the batch rows
  // weight-gradient GEMMs: one CTA per SM (TMEM-bound), the rows split evenly
  const int sms = sm_count();
  const int per_split = max(8, (kb_rows + min(sms, kMaxSplits) - 1) / min(sms, kMaxSplits));
  const int splits = (kb_rows + per_split - 1) / per_split;  // <= kMaxSplits
  float* part = ptr<float>(ws, L.off_part);

  // bias gradient of a layer: column K of its dW block
  auto dbias_of = [&](int l) { return dwx + dwx_off(l) + (l == 0 ? kIn : kW); };
  auto ldb_of = [&](int l) { return (l == 0 ? kIn : kW) + kExt; };
  const bool inj_loads = g_inject.load(std::memory_order_relaxed) == 1;
  const unsigned long long wait_ns = inj_loads ? 50000000ull : 2000000000ull;
  mlp_head_grad_kernel<<<(Mp + 127) / 128, 128, 0, st>>>(d_delta, L.M, Mp, dzh, dzht,
                                                         dbias_of(kDepth), kW + kExt);
  count_launches(1);
  // head: dW_head += dZh^T H_7 (H_7 read MN-major)
  {
    CUtensorMap ma, mb;
    if (!make_map(&ma, dzht, kHeadRows, Mp, Mp, BM) ||
        !make_map(&mb, H(kDepth - 1), Mp, kW, kW, BK))
      return GFTORF_ERR_CUDA;
    GemmArgs a;
    memset(&a, 0, sizeof(a));
    a.kb_total = kb_rows, a.kb_per_split = per_split;
    a.rows_valid = 3, a.cols_valid = kW;
    a.out_f = dwx + dwx_off(kDepth), a.ldf = kW + kExt;
    a.status = status, a.inject_no_loads = inj_loads, a.wait_ns = wait_ns;
    if (!gemm<256, EPI_ATOMIC, 1, 0, 1>(ma, mb, a, 1, 1, splits, st)) return GFTORF_ERR_CUDA;
  }
  if (g_inject.load(std::memory_order_relaxed) != 2) {
    // fused dZ chain: all layers per pair of 128-row tiles, dZ_l kept in
    // shared memory as the next layer's operand and stored (row-major) for
    // the weight gradients below
    if (!fused_configured()) return GFTORF_ERR_CUDA;
    FusedMaps maps;
    if (!make_map(&maps.w[kDepth], wt + wb_off(kDepth), kW, kHeadRows, kHeadRows, 256))
      return GFTORF_ERR_CUDA;
    for (int l = 0; l < kDepth; ++l)
      if (!make_map(&maps.w[l], wt + wb_off(l), l == 0 ? kIn : kW, kW, kW, 256))
        return GFTORF_ERR_CUDA;
    if (!make_map(&maps.act, dz(0), (uint64_t)kDepth * Mp, kW, kW, BM)) return GFTORF_ERR_CUDA;
    FusedBwdArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.dd = d_delta, fa.bits = bits, fa.denc = denc;
    fa.M = L.M, fa.Mp = Mp, fa.n_tiles = mt;
    const int n_pairs = (mt + kPair - 1) / kPair;
    mlp_fused_bwd_kernel<<<n_pairs < sms ? n_pairs : sms, kFusedThreads, kBwdSmem, st>>>(
        maps, fa, status, wait_ns, inj_loads);
    count_launches(1);
  } else {
    // dH_7 = dZh W_head, dZ_7 = dH_7 * (H_7 > 0); then dH_{l-1} = dZ_l W_l
    // (l = 0: the encoding's gradient, FP32), one GEMM per layer
    for (int l = kDepth; l >= 1; --l) {
      const int K = l == kDepth ? kHeadRows : kW;
      CUtensorMap ma, mb;
      if (!make_map(&ma, l == kDepth ? dzh : dz(l), Mp, K, K, BM) ||
          !make_map(&mb, wt + wb_off(l), l == 0 ? kIn : kW, K, K, 256))
        return GFTORF_ERR_CUDA;
      GemmArgs a;
      memset(&a, 0, sizeof(a));
      a.kb_total = l == kDepth ? 1 : kW / BK, a.kb_per_split = a.kb_total;
      a.rows_valid = Mp, a.cols_valid = kW;
      a.out_b = dz(l - 1), a.ldo = kW;
      a.mbits = bits + (size_t)(l - 1) * Mp * (kW / 32);
      a.status = status, a.inject_no_loads = inj_loads, a.wait_ns = wait_ns;
      if (!gemm<256, EPI_MASK>(ma, mb, a, mt, 1, 1, st)) return GFTORF_ERR_CUDA;
    }
    CUtensorMap ma, mb;
    if (!make_map(&ma, dz(0), Mp, kW, kW, BM) || !make_map(&mb, wt, kIn, kW, kW, 256))
      return GFTORF_ERR_CUDA;
    GemmArgs a;
    memset(&a, 0, sizeof(a));
    a.kb_total = kW / BK, a.kb_per_split = kW / BK;
    a.rows_valid = Mp, a.cols_valid = kIn;
    a.out_f = denc, a.ldf = kIn;
    a.status = status, a.inject_no_loads = inj_loads, a.wait_ns = wait_ns;
    if (!gemm<256, EPI_F32>(ma, mb, a, mt, 1, 1, st)) return GFTORF_ERR_CUDA;
  }
  // dW_l += dZ_l^T H_{l-1} (or the encoding): all 256 output rows per CTA,
  // both operands read MN-major from the row-major dZ_l and H_{l-1}
  for (int l = kDepth - 1; l >= 0; --l) {
    const int K = l == 0 ? kIn : kW;
    CUtensorMap ma, mb;
    if (!make_map(&ma, dz(l), Mp, kW, kW, BK) ||
        !make_map(&mb, l == 0 ? enc : H(l - 1), Mp, K, K, BK))
      return GFTORF_ERR_CUDA;
    GemmArgs a;
    memset(&a, 0, sizeof(a));
    a.kb_total = kb_rows, a.kb_per_split = per_split;
    a.rows_valid = kW, a.cols_valid = K;
    a.out_f = part, a.ldf = K;
    a.dbias = dbias_of(l), a.ldb = ldb_of(l);  // the column sums of dZ_l
    a.status = status, a.inject_no_loads = inj_loads, a.wait_ns = wait_ns;
    if (!(l == 0 ? gemm<kIn, EPI_PARTIAL, 2, 1, 1>(ma, mb, a, 1, 1, splits, st)
                 : gemm<kW, EPI_PARTIAL, 2, 1, 1>(ma, mb, a, 1, 1, splits, st)))
      return GFTORF_ERR_CUDA;
    mlp_reduce_dw_kernel<<<(kW * K + 255) / 256, 256, 0, st>>>(part, splits, K, dwx + dwx_off(l),
                                                               K + kExt);
    count_launches(1);
  }
  mlp_unpack_grads_kernel<<<4 * 152, 256, 0, st>>>(dwx, d_theta);
  mlp_encode_bwd_kernel<<<(n_gaussians + 7) / 8, 256, 0, st>>>(means, denc, n_gaussians,
                                                               n_frames, inv_scale, d_means);
  count_launches(2);
  (void)times;
  return cudaGetLastError() == cudaSuccess ? GFTORF_OK : GFTORF_ERR_CUDA;
}

extern "C" gftorf_status gftorf_mlp_read_status(void* workspace, size_t workspace_bytes,
                                                void* stream) {
  if (!workspace || workspace_bytes < 256) return GFTORF_ERR_WORKSPACE;
  int s = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&s, workspace, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GFTORF_ERR_CUDA;
  return (gftorf_status)s;
}

extern "C" gftorf_status gftorf_mlp_export(int32_t n_gaussians, int32_t n_frames, int32_t what,
                                           int32_t layer, void* dst, void* workspace,
                                           size_t workspace_bytes, void* stream) {
  if (!mlp_args_ok(n_gaussians, n_frames) || !dst) return GFTORF_ERR_ARG;
  const MlpLayout L = mlp_layout(n_gaussians, n_frames);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 ||
      workspace_bytes < L.total)
    return GFTORF_ERR_WORKSPACE;
  const size_t Mp = (size_t)L.M_pad, M = (size_t)L.M;
  size_t off, bytes;
  if ((what == 1 || what == 2) && (layer < 0 || layer >= kDepth)) return GFTORF_ERR_ARG;
  switch (what) {
    case 0: off = L.off_enc, bytes = M * kIn * 2; break;
    case 1: off = L.off_h + (size_t)layer * Mp * kW * 2, bytes = M * kW * 2; break;
    case 2: off = L.off_dz + (size_t)layer * Mp * kW * 2, bytes = M * kW * 2; break;
    case 3: off = L.off_denc, bytes = M * kIn * 4; break;
    default: return GFTORF_ERR_ARG;
  }
  if (bytes == 0) return GFTORF_OK;
  const cudaError_t e =
      cudaMemcpyAsync(dst, static_cast<unsigned char*>(workspace) + off, bytes,
                      cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GFTORF_OK : GFTORF_ERR_CUDA;
}

extern "C" void gftorf_mlp_debug_inject(int32_t mode) {
  g_inject.store(mode == 1 || mode == 2 ? mode : 0, std::memory_order_relaxed);
}

extern "C" gftorf_status gftorf_mlp_infer(int32_t n_gaussians, int32_t n_frames,
                                          const float* theta, const float* means,
                                          const float* times, float inv_scale, float* delta,
                                          void* workspace, size_t workspace_bytes, void* stream) {
  gftorf::TraceRange trace_("gftorf_mlp_infer");
  if (!mlp_args_ok(n_gaussians, n_frames) || !theta || !times ||
      (n_gaussians > 0 && (!means || !delta)) || !(inv_scale > 0.f))
    return GFTORF_ERR_ARG;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0 ||
      workspace_bytes < gftorf_mlp_infer_workspace_size())
    return GFTORF_ERR_WORKSPACE;
  for (int b = 0; b < n_frames; ++b)
    if (!std::isfinite(times[b])) return GFTORF_ERR_ARG;
  if (!encode_fn()) return GFTORF_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* status = ptr<int>(workspace, 0);
  cudaMemsetAsync(status, 0, 256, st);
  const int M = n_gaussians * n_frames;
  if (M == 0) return cudaGetLastError() == cudaSuccess ? GFTORF_OK : GFTORF_ERR_CUDA;
  auto* wb = ptr<__nv_bfloat16>(workspace, 256);
  auto* wt = wb + wb_elems();
  mlp_prep_weights_kernel<<<4 * 152, 256, 0, st>>>(theta, wb, wt);
  FusedMaps maps;
  for (int l = 0; l <= kDepth; ++l) {
    const int K = l == 0 ? kIn : kW, rows = l == kDepth ? kHeadRows : kW;
    if (!make_map(&maps.w[l], wb + wb_off(l), rows, K, K, rows)) return GFTORF_ERR_CUDA;
  }
  Times tm;
  memset(&tm, 0, sizeof(tm));
  for (int b = 0; b < n_frames; ++b) tm.t[b] = times[b];
  if (!fused_configured()) return GFTORF_ERR_CUDA;
  const int sms = sm_count();
  const int n_tiles = (M + BM - 1) / BM;
  const int n_pairs = (n_tiles + kPair - 1) / kPair;
  const unsigned long long wait_ns = g_inject.load() == 1 ? 50000000ull : 2000000000ull;
  FusedKeep none;
  memset(&none, 0, sizeof(none));
  mlp_fused_fwd_kernel<false><<<n_pairs < sms ? n_pairs : sms, kFusedThreads, kFusedSmem, st>>>(
      maps, theta, means, tm, n_gaussians, M, n_tiles, inv_scale, delta, status, wait_ns,
      g_inject.load() == 1, none);
  count_launches(2);
  return cudaGetLastError() == cudaSuccess ? GFTORF_OK : GFTORF_ERR_CUDA;
}
