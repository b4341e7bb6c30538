// S-parameter surrogate: BF16 tcgen05 GEMMs with FP32 accumulation in tensor memory, and
// the small kernels around them (input mapping, loss, bias gradients, Adam, ensemble gate).
//
// Every matrix product of the network, forward and backward, is one shape:
//   C[P x Q] = sum_r A[p, r] B[q, r]          (A: P x R, B: Q x R, both row-major BF16)
// i.e. both operands K-major.  The three products of a layer map onto it as
//   forward   z = a W^T        A = a      [batch x in],  B = W   [out x in]
//   dgrad     da = dz W        A = dz     [batch x out], B = W^T [in x out]
//   wgrad     dW = dz^T a      A = dz^T   [out x batch], B = a^T [in x batch]
// so the epilogues that produce a and dz also write their transposes.
//
// k_mlp_gemm: one 128 x NT output tile per CTA.  Warp 0 (one lane) streams 64-wide K slices
// of A and B into a ring of shared-memory stages with TMA (128-byte swizzle); warp 1 owns the
// tensor-memory allocation and (one lane) issues tcgen05.mma (M = 128, N = NT, K = 16) on the
// staged slices, releasing each stage with tcgen05.commit; warps 2..9 wait for the final
// commit, read the FP32 accumulator with tcgen05.ld (each warp half the columns of its 32-lane
// quarter) and run the epilogue.  Every mbarrier wait is bounded (2 s of %globaltimer); a wait that gives up
// sets bit 1 of the status word and the block drains and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "yf_internal.h"
#include "yfmlp.h"

namespace yf {
namespace mlp {

using bf16 = __nv_bfloat16;

constexpr int kIn = YF_MLP_IN, kWidth = YF_MLP_WIDTH, kOut = YF_MLP_OUT, kLayers = YF_MLP_LAYERS;
constexpr int kK1 = 64;        // layer-1 K padded to one 64-wide slice (6 real columns)
constexpr int kBM = 128;       // rows per tile (tcgen05 M)
constexpr int kBK = 64;        // K per stage: 64 BF16 = one 128-byte swizzle row
constexpr int kEpiWarps = 8;   // two per 32-lane quarter of the accumulator, half the columns each
constexpr int kThreads = 64 + 32 * kEpiWarps;   // producer warp, MMA warp, epilogue warps
constexpr long kParams = YF_MLP_PARAMS;

// flat parameter offsets: W_l [out][in] then b_l [out]
__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? kIn : kWidth; }
__host__ __device__ constexpr long w_off(int l)
{
    return l == 0 ? 0 : (long)kWidth * kIn + kWidth + (long)(l - 1) * ((long)kWidth * kWidth + kWidth);
}
__host__ __device__ constexpr long b_off(int l) { return w_off(l) + (long)kWidth * layer_in(l); }
static_assert(b_off(kLayers - 1) + kOut == kParams, "parameter count");

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: gives up after 2 s or when another role of the block has given up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (gtimer() - t0 > 2000000000ull) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// bulk tensor store of a staged box (shared -> global), tracked by the thread's bulk group
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, uint32_t src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// this thread's bulk stores have read their shared sources / are complete
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand staged by TMA with the 128-byte
// swizzle: rows of 128 bytes (64 BF16 of K), 8-row groups 1024 bytes apart (stride byte
// offset), descriptor version 1, swizzle mode 2 (128 B).  The leading byte offset is not used
// by swizzled K-major layouts.  Advancing K by 16 elements inside the 128-byte row adds 32
// bytes to the start address; the hardware applies the swizzle to the resulting address,
// which is why stage bases are 1024-byte aligned.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 lanes x 32 consecutive FP32 columns: thread t of the warp gets lane (base lane + t)
// 32 columns of one accumulator row per thread, without waiting: the registers are valid only
// after tmem_wait32 on the same array
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// wait for this thread's outstanding TMEM loads; the array is an operand so that no use of it
// is scheduled before the wait
__device__ __forceinline__ void tmem_wait32(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]),
                   "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]),
                   "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// gelu in its tanh form and its derivative; tanh by the hardware approximation instruction
__device__ __forceinline__ float tanh_hw(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kGeluC = 0.7978845608028654f;   // sqrt(2 / pi)
constexpr float kGeluA = 0.044715f;
__device__ __forceinline__ float gelu(float x)
{
    const float th = tanh_hw(kGeluC * (x + kGeluA * x * x * x));
    return 0.5f * x * (1.f + th);
}
// the same on a pair of values through the paired FP32 instructions: (kA x) x, then
// fma(., x, x), times kC; 0.5 x (1 + tanh)
__device__ __forceinline__ float2 gelu2(float2 x)
{
    const float2 u = __fmul2_rn(make_float2(kGeluC, kGeluC),
                                __ffma2_rn(__fmul2_rn(__fmul2_rn(make_float2(kGeluA, kGeluA), x), x), x, x));
    const float2 s = __fadd2_rn(make_float2(1.f, 1.f), make_float2(tanh_hw(u.x), tanh_hw(u.y)));
    return __fmul2_rn(__fmul2_rn(make_float2(0.5f, 0.5f), x), s);
}
__device__ __forceinline__ float gelu_grad(float x)
{
    const float th = tanh_hw(kGeluC * (x + kGeluA * x * x * x));
    return 0.5f * (1.f + th) + 0.5f * x * (1.f - th * th) * kGeluC * (1.f + 3.f * kGeluA * x * x);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// ------------------------------------------------------------------ GEMM

enum { MODE_HIDDEN = 0, MODE_OUT = 1, MODE_DGRAD = 2, MODE_WGRAD = 3 };

struct GemmArgs {
    int P, Q, R;             // C[P x Q] = A[P x R] B[Q x R]^T; P % 128 == 0, Q % NT == 0, R % 64 == 0
    int a_row0, b_row0;      // row offsets of the operands inside their tensor maps
    int mode;
    const float *bias;       // [Q]                   HIDDEN, OUT
    float *out_f32;          // z (HIDDEN, nullable), y (OUT), dW (WGRAD); row stride ld_f32
    int ld_f32;
    bf16 *out_bf;            // a (HIDDEN) or dz (DGRAD), row-major, nullable; row stride ld_bf
    int ld_bf;
    bf16 *out_t;             // its transpose [Q][P], nullable; row stride ld_t
    int ld_t;
    const float *zin;        // pre-activations (DGRAD); row stride ld_z
    int ld_z;
    int qvalid;              // WGRAD: only columns < qvalid are written
    int *status;
    int tma_store;           // inference (persistent kernel): a (HIDDEN) or y (OUT) stored by TMA through the store map
    int out_row0;            // OUT with tma_store: row of y's first row in the store map
};

// Epilogue of 32 accumulator columns of one row: r = FP32 accumulator values of row `row`,
// columns q .. q + 31 of C.
__device__ __forceinline__ void epi_chunk(const GemmArgs &g, const uint32_t (&r)[32], int row, int q,
                                          const float *bias)
{
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
    if (g.mode == MODE_HIDDEN || g.mode == MODE_OUT) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 b4 = reinterpret_cast<const float4 *>(bias + q)[i];
            v[4 * i] += b4.x; v[4 * i + 1] += b4.y; v[4 * i + 2] += b4.z; v[4 * i + 3] += b4.w;
        }
        if (g.out_f32) {
            float4 *o = (float4 *)(g.out_f32 + (size_t)row * g.ld_f32 + q);
#pragma unroll
            for (int i = 0; i < 8; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
        if (g.mode == MODE_OUT) return;
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = gelu(v[i]);
    } else if (g.mode == MODE_DGRAD) {
        const float4 *zr = (const float4 *)(g.zin + (size_t)row * g.ld_z + q);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 z4 = __ldg(zr + i);
            v[4 * i + 0] *= gelu_grad(z4.x);
            v[4 * i + 1] *= gelu_grad(z4.y);
            v[4 * i + 2] *= gelu_grad(z4.z);
            v[4 * i + 3] *= gelu_grad(z4.w);
        }
    } else {   // WGRAD
        float *o = g.out_f32 + (size_t)row * g.ld_f32;
        if (q + 32 <= g.qvalid && (g.ld_f32 & 3) == 0) {
            float4 *o4 = (float4 *)(o + q);
#pragma unroll
            for (int i = 0; i < 8; ++i) o4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        } else {
            for (int i = 0; i < 32; ++i)
                if (q + i < g.qvalid) o[q + i] = v[i];
        }
        return;
    }
    // BF16 row-major copy and transpose (HIDDEN: a, DGRAD: dz)
    if (g.out_bf) {
        uint4 *o = (uint4 *)(g.out_bf + (size_t)row * g.ld_bf + q);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            o[i] = make_uint4(pack_bf16(v[8 * i + 0], v[8 * i + 1]), pack_bf16(v[8 * i + 2], v[8 * i + 3]),
                              pack_bf16(v[8 * i + 4], v[8 * i + 5]), pack_bf16(v[8 * i + 6], v[8 * i + 7]));
    }
    if (g.out_t) {
#pragma unroll
        for (int i = 0; i < 32; ++i) g.out_t[(size_t)(q + i) * g.ld_t + row] = __float2bfloat16_rn(v[i]);
    }
}

// Hidden-layer epilogue with only the BF16 activations to write (the inference path): bias,
// GELU, then the warp's 32 x 32 chunk goes through its shared-memory staging area (rows of
// 80 bytes: a quarter-warp's 16-byte writes hit distinct banks) so that each global store
// instruction writes 8 rows of 64 contiguous bytes instead of 32 rows of 16.
constexpr int kStageRow = 80;
__device__ __forceinline__ void epi_hidden_staged(const GemmArgs &g, const uint32_t (&r)[32], int row0, int lane,
                                                  int q, const float *bias, uint8_t *stg)
{
    float v[32];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 b4 = reinterpret_cast<const float4 *>(bias + q)[i];
        const float2 a = gelu2(__fadd2_rn(make_float2(__uint_as_float(r[4 * i]), __uint_as_float(r[4 * i + 1])),
                                          make_float2(b4.x, b4.y)));
        const float2 b = gelu2(__fadd2_rn(make_float2(__uint_as_float(r[4 * i + 2]), __uint_as_float(r[4 * i + 3])),
                                          make_float2(b4.z, b4.w)));
        v[4 * i] = a.x;
        v[4 * i + 1] = a.y;
        v[4 * i + 2] = b.x;
        v[4 * i + 3] = b.y;
    }
    uint4 *srow = reinterpret_cast<uint4 *>(stg + lane * kStageRow);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        srow[j] = make_uint4(pack_bf16(v[8 * j + 0], v[8 * j + 1]), pack_bf16(v[8 * j + 2], v[8 * j + 3]),
                             pack_bf16(v[8 * j + 4], v[8 * j + 5]), pack_bf16(v[8 * j + 6], v[8 * j + 7]));
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int rr = 8 * k + (lane >> 2), cc = lane & 3;
        const uint4 val = *reinterpret_cast<const uint4 *>(stg + rr * kStageRow + cc * 16);
        *reinterpret_cast<uint4 *>(g.out_bf + (size_t)(row0 + rr) * g.ld_bf + q + 8 * cc) = val;
    }
    __syncwarp();
}

// The same epilogue with the 32 x 32 BF16 chunk written by a bulk tensor store: the warp fills its
// 2 KB stage (rows of 64 bytes, 16-byte units placed by the 64-byte swizzle of the store map,
// unit u of row r at u ^ ((r >> 1) & 3), so that a quarter-warp's row writes hit distinct banks)
// and lane 0 issues the store.  The stage is refilled only after the previous store has read it.
__device__ __forceinline__ void epi_hidden_tma(const CUtensorMap *tc, const uint32_t (&r)[32], int row0, int lane,
                                               int q, const float *bias, uint8_t *stg)
{
    uint32_t pk[16];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 b4 = reinterpret_cast<const float4 *>(bias + q)[i];
        const float2 a = gelu2(__fadd2_rn(make_float2(__uint_as_float(r[4 * i]), __uint_as_float(r[4 * i + 1])),
                                          make_float2(b4.x, b4.y)));
        const float2 b = gelu2(__fadd2_rn(make_float2(__uint_as_float(r[4 * i + 2]), __uint_as_float(r[4 * i + 3])),
                                          make_float2(b4.z, b4.w)));
        pk[2 * i] = pack_bf16(a.x, a.y);
        pk[2 * i + 1] = pack_bf16(b.x, b.y);
    }
    if (lane == 0) bulk_wait_read();
    __syncwarp();
    const int sw = (lane >> 1) & 3;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        *reinterpret_cast<uint4 *>(stg + lane * 64 + ((j ^ sw) << 4)) =
            make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) tma_store_2d(tc, q, row0, smem_u32(stg));
}

// Output-layer epilogue (bias, FP32 y only): the same staging, one 16-column half of the
// chunk at a time (64 bytes of a row each)
__device__ __forceinline__ void epi_out_staged(const GemmArgs &g, const uint32_t (&r)[32], int row0, int lane,
                                               int q, const float *bias, uint8_t *stg)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint4 *srow = reinterpret_cast<uint4 *>(stg + lane * kStageRow);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 16 * h + 4 * j;
            const float4 b4 = *reinterpret_cast<const float4 *>(bias + q + c);
            srow[j] = make_uint4(__float_as_uint(__uint_as_float(r[c]) + b4.x),
                                 __float_as_uint(__uint_as_float(r[c + 1]) + b4.y),
                                 __float_as_uint(__uint_as_float(r[c + 2]) + b4.z),
                                 __float_as_uint(__uint_as_float(r[c + 3]) + b4.w));
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int rr = 8 * k + (lane >> 2), cc = lane & 3;
            const uint4 val = *reinterpret_cast<const uint4 *>(stg + rr * kStageRow + cc * 16);
            *reinterpret_cast<uint4 *>(g.out_f32 + (size_t)(row0 + rr) * g.ld_f32 + q + 16 * h + 4 * cc) = val;
        }
        __syncwarp();
    }
}

// Output-layer epilogue through the bulk stores: each 16-column half of the chunk (64 bytes of a
// row, FP32) goes through the warp's 2 KB stage with the same 64-byte swizzle as above.
__device__ __forceinline__ void epi_out_tma(const CUtensorMap *tc, const uint32_t (&r)[32], int row0, int lane,
                                           int q, const float *bias, uint8_t *stg)
{
    const int sw = (lane >> 1) & 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint4 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 16 * h + 4 * j;
            const float4 b4 = *reinterpret_cast<const float4 *>(bias + q + c);
            v[j] = make_uint4(__float_as_uint(__uint_as_float(r[c]) + b4.x),
                              __float_as_uint(__uint_as_float(r[c + 1]) + b4.y),
                              __float_as_uint(__uint_as_float(r[c + 2]) + b4.z),
                              __float_as_uint(__uint_as_float(r[c + 3]) + b4.w));
        }
        if (lane == 0) bulk_wait_read();
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 4; ++j) *reinterpret_cast<uint4 *>(stg + lane * 64 + ((j ^ sw) << 4)) = v[j];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) tma_store_2d(tc, q + 16 * h, row0, smem_u32(stg));
    }
}

template <int NT, int kStages>
struct GemmSmem {
    static constexpr int A_BYTES = kBM * kBK * 2;            // 16 KB
    static constexpr int B_BYTES = NT * kBK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int BAR_OFF = kStages * STAGE;
    static constexpr int BYTES = BAR_OFF + 128 + 1024;        // barriers, slots, alignment slack
    static constexpr uint32_t TMEM_COLS = NT < 32 ? 32 : NT;
};

template <int NT, int kStages>
__global__ void __launch_bounds__(kThreads, 2)
k_mlp_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, GemmArgs g)
{
    using S = GemmSmem<NT, kStages>;
    extern __shared__ uint8_t smem_raw[];
    // stage bases 1024-byte aligned in the shared window (the 128-byte swizzle repeats every
    // 8 rows of 128 bytes and is computed from the address bits)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *sm = smem_raw + (sbase - raw);
    uint64_t *bars = (uint64_t *)(sm + S::BAR_OFF);   // full[kStages], empty[kStages], done
    volatile uint32_t *tmem_slot = (volatile uint32_t *)(sm + S::BAR_OFF + 8 * (2 * kStages + 1));
    volatile int *abort = (volatile int *)(tmem_slot + 1);
    volatile int *consumed = (volatile int *)(tmem_slot + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p0 = blockIdx.x * kBM, q0 = blockIdx.y * NT;
    const int nk = g.R / kBK;
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[kStages + s]); };
    const uint32_t done = smem_u32(&bars[2 * kStages]);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(done, 1);
        *abort = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void *)tmem_slot)),
                     "r"(S::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kc = 0; kc < nk; ++kc) {
                const int s = kc % kStages;
                if (kc >= kStages && !mbar_wait(empty(s), ((kc / kStages) - 1) & 1, abort)) {
                    *abort = 1;
                    atomicOr(g.status, 2);
                    break;
                }
                const uint32_t a_dst = sbase + s * S::STAGE, b_dst = a_dst + S::A_BYTES;
                mbar_expect_tx(full(s), S::STAGE);
                tma_load_2d(a_dst, &ta, kc * kBK, g.a_row0 + p0, full(s));
                tma_load_2d(b_dst, &tb, kc * kBK, g.b_row0 + q0, full(s));
                ++issued;
            }
            if (*abort) {
                // let the copies already in flight land before the block's memory is released
                volatile int keep_waiting = 0;
                for (int kc = *consumed; kc < issued; ++kc)
                    mbar_wait(full(kc % kStages), (kc / kStages) & 1, &keep_waiting);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(kBM, NT);
            for (int kc = 0; kc < nk; ++kc) {
                const int s = kc % kStages;
                if (!mbar_wait(full(s), (kc / kStages) & 1, abort)) {
                    *abort = 1;
                    atomicOr(g.status, 2);
                    break;
                }
                tc_fence_after();
                const uint32_t a_s = sbase + s * S::STAGE, b_s = a_s + S::A_BYTES;
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k)
                    mma_bf16(tmem, sw128_desc(a_s + 32 * k), sw128_desc(b_s + 32 * k), idesc,
                             (kc | k) != 0);
                mma_commit(empty(s));
                *consumed = kc + 1;
            }
            mma_commit(done);   // also on abort: arrives once the issued MMAs have finished
        }
    } else {
        const bool ok = mbar_wait(done, 0, abort);
        tc_fence_after();
        if (!ok) {
            *abort = 1;
            atomicOr(g.status, 2);
        }
        // warp w may read TMEM lanes 32 (w % 4) .. +31; the two warps of a quarter split the
        // columns
        const int qtr = warp & 3, half = (warp - 2) >> 2;
        constexpr int NCOL = NT / 2;
        const int row = p0 + 32 * qtr + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * qtr) << 16);
        // tcgen05.ld is warp-collective: the loop condition must be the same on all lanes
        for (int c0 = half * NCOL; c0 < (half + 1) * NCOL && __all_sync(0xffffffffu, ok && !*abort); c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tl + c0, r);
            epi_chunk(g, r, row, q0 + c0, g.bias);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(S::TMEM_COLS)
                     : "memory");
    }
}

// Persistent form for large grids: one CTA per SM loops over output tiles (row-block major,
// so the two column tiles of a row block run back to back and share A through L2).  Two FP32
// accumulators of NT columns live in TMEM: the producer and MMA warps move on to tile t+1
// while the eight epilogue warps drain tile t, and the MMA warp reuses an accumulator only
// after all epilogue warps have released it (tmem_empty).  Same operands, epilogue and
// results as k_mlp_gemm.
template <int NT>
struct PersistSmem {
    static constexpr int ST = 4;
    static constexpr int A_BYTES = kBM * kBK * 2;
    static constexpr int B_BYTES = NT * kBK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int BAR_OFF = ST * STAGE;
    static constexpr int NBAR = 2 * ST + 5;     // full, empty, tmem_full[2], tmem_empty[2], drain
    // bias of all Q <= 512 columns, read as float4: 16-byte (here 128-byte) aligned
    static constexpr int BIAS_OFF = (BAR_OFF + 8 * NBAR + 64 + 127) / 128 * 128;
    // per epilogue warp: its staging rows (epi_hidden_staged, epi_out_staged: 32 rows of 80 bytes;
    // epi_hidden_tma: a 2 KB stage, 512-byte aligned for the store map's 64-byte swizzle)
    static constexpr int STG_STRIDE = 3072;
    static constexpr int STG_OFF = (BIAS_OFF + 4 * 512 + 1023) / 1024 * 1024;
    static constexpr int BYTES = STG_OFF + kEpiWarps * STG_STRIDE + 1024;
    static_assert(STG_STRIDE >= 32 * kStageRow && STG_STRIDE % 512 == 0, "staging per warp");
    static_assert(STG_OFF % 16 == 0, "16-byte staging writes");
    static_assert(BYTES <= 227 * 1024, "shared memory of one CTA");
    static_assert(BIAS_OFF % 16 == 0, "float4 reads of the staged bias");
    static constexpr uint32_t TMEM_COLS = 2 * NT;
    static_assert(2 * NT <= 512, "two accumulators must fit the 512 TMEM columns");
};

// the hidden-layer inference epilogue writes through the store map (the host sets tma_store only
// with a map of the output buffer)
__device__ __forceinline__ bool staged_tma_ok(const GemmArgs &g)
{
    return g.tma_store && g.mode == MODE_HIDDEN && g.out_bf && !g.out_f32 && !g.out_t && g.bias;
}
// the output-layer inference epilogue writes y through the store map; out_row0 is the first row of
// this GEMM's y inside that map
__device__ __forceinline__ bool out_tma_ok(const GemmArgs &g)
{
    return g.tma_store && g.mode == MODE_OUT && g.out_f32 && g.bias;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int NT>
__global__ void __launch_bounds__(kThreads, 1)
k_mlp_gemm_persist(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                   const __grid_constant__ CUtensorMap tc, GemmArgs g)
{
    using S = PersistSmem<NT>;
    constexpr int ST = S::ST;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *sm = smem_raw + (sbase - raw);
    uint64_t *bars = (uint64_t *)(sm + S::BAR_OFF);
    volatile uint32_t *tmem_slot = (volatile uint32_t *)(sm + S::BAR_OFF + 8 * S::NBAR);
    volatile int *abort = (volatile int *)(tmem_slot + 1);
    volatile int *consumed = (volatile int *)(tmem_slot + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntn = g.Q / NT, ntiles = (g.P / kBM) * ntn;
    const int nk = g.R / kBK;
    auto full = [&](int s) { return smem_u32(&bars[s]); };
    auto empty = [&](int s) { return smem_u32(&bars[ST + s]); };
    auto tfull = [&](int b) { return smem_u32(&bars[2 * ST + b]); };
    auto tempty = [&](int b) { return smem_u32(&bars[2 * ST + 2 + b]); };
    const uint32_t drain = smem_u32(&bars[2 * ST + 4]);

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull(b), 1);
            mbar_init(tempty(b), kEpiWarps);
        }
        mbar_init(drain, 1);
        *abort = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void *)tmem_slot)),
                     "r"(S::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    auto give_up = [&]() {
        *abort = 1;
        atomicOr(g.status, 2);
    };

    if (warp == 0) {
        if (lane == 0) {
            int c = 0;   // running slice count of this CTA: stage c % ST, use c / ST
            for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
                const int p0 = (t / ntn) * kBM, q0 = (t % ntn) * NT;
                for (int kc = 0; kc < nk; ++kc, ++c) {
                    const int s = c % ST;
                    if (c >= ST && !mbar_wait(empty(s), ((c / ST) - 1) & 1, abort)) {
                        give_up();
                        break;
                    }
                    const uint32_t a_dst = sbase + s * S::STAGE, b_dst = a_dst + S::A_BYTES;
                    mbar_expect_tx(full(s), S::STAGE);
                    tma_load_2d(a_dst, &ta, kc * kBK, g.a_row0 + p0, full(s));
                    tma_load_2d(b_dst, &tb, kc * kBK, g.b_row0 + q0, full(s));
                }
            }
            if (*abort) {
                // slices issued but never consumed: let their copies land before exit
                volatile int keep_waiting = 0;
                for (int k = *consumed; k < c; ++k) mbar_wait(full(k % ST), (k / ST) & 1, &keep_waiting);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(kBM, NT);
            int c = 0, it = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x, ++it) {
                const int b = it & 1;
                if (it >= 2 && !mbar_wait(tempty(b), ((it >> 1) - 1) & 1, abort)) {
                    give_up();
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * NT);
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++c) {
                    const int s = c % ST;
                    if (!mbar_wait(full(s), (c / ST) & 1, abort)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_s = sbase + s * S::STAGE, b_s = a_s + S::A_BYTES;
#pragma unroll
                    for (int k = 0; k < kBK / 16; ++k)
                        mma_bf16(acc, sw128_desc(a_s + 32 * k), sw128_desc(b_s + 32 * k), idesc, (kc | k) != 0);
                    mma_commit(empty(s));
                    *consumed = c + 1;
                }
                if (!ok) break;
                mma_commit(tfull(b));
            }
            // every MMA issued so far has completed once this arrives; TMEM may then be freed
            mma_commit(drain);
            volatile int keep_waiting = 0;
            mbar_wait(drain, 0, &keep_waiting);
        }
    } else {
        const int qtr = warp & 3, half = (warp - 2) >> 2;
        constexpr int NCOL = NT / 2;
        // the layer's bias, once per CTA, for every tile's epilogue (named barrier 1: the
        // epilogue warps only)
        float *sbias = reinterpret_cast<float *>(sm + S::BIAS_OFF);
        uint8_t *stg = sm + S::STG_OFF + (warp - 2) * S::STG_STRIDE;
        const bool tstore = staged_tma_ok(g), ostore = out_tma_ok(g);
        const bool staged = g.mode == MODE_HIDDEN && g.out_bf && !g.out_f32 && !g.out_t && g.bias;
        const bool staged_out = g.mode == MODE_OUT && g.out_f32 && g.bias && (g.ld_f32 & 3) == 0;
        if (g.bias)
            for (int c = threadIdx.x - 64; c < g.Q; c += 32 * kEpiWarps) sbias[c] = __ldg(g.bias + c);
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
        int it = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int b = it & 1;
            const bool ok = mbar_wait(tfull(b), (it >> 1) & 1, abort);
            if (__any_sync(0xffffffffu, !ok)) {
                if (lane == 0) give_up();
                break;
            }
            tc_fence_after();
            const int p0 = (t / ntn) * kBM, q0 = (t % ntn) * NT;
            const int row = p0 + 32 * qtr + lane;
            const uint32_t tl = tmem + ((uint32_t)(32 * qtr) << 16) + (uint32_t)(b * NT);
            // the next 32 columns load from TMEM while this chunk's epilogue runs
            static_assert(NCOL % 64 == 0, "chunks are processed in pairs");
            uint32_t ra[32], rb[32];
            const int cb = half * NCOL;
            tmem_ld32_async(tl + cb, ra);
            tmem_wait32(ra);
            for (int c0 = cb; c0 < cb + NCOL; c0 += 64) {
                tmem_ld32_async(tl + c0 + 32, rb);
                if (tstore) epi_hidden_tma(&tc, ra, p0 + 32 * qtr, lane, q0 + c0, sbias, stg);
                else if (staged) epi_hidden_staged(g, ra, p0 + 32 * qtr, lane, q0 + c0, sbias, stg);
                else if (ostore) epi_out_tma(&tc, ra, g.out_row0 + p0 + 32 * qtr, lane, q0 + c0, sbias, stg);
                else if (staged_out) epi_out_staged(g, ra, p0 + 32 * qtr, lane, q0 + c0, sbias, stg);
                else epi_chunk(g, ra, row, q0 + c0, sbias);
                tmem_wait32(rb);
                if (c0 + 64 < cb + NCOL) tmem_ld32_async(tl + c0 + 64, ra);
                if (tstore) epi_hidden_tma(&tc, rb, p0 + 32 * qtr, lane, q0 + c0 + 32, sbias, stg);
                else if (staged) epi_hidden_staged(g, rb, p0 + 32 * qtr, lane, q0 + c0 + 32, sbias, stg);
                else if (ostore) epi_out_tma(&tc, rb, g.out_row0 + p0 + 32 * qtr, lane, q0 + c0 + 32, sbias, stg);
                else if (staged_out) epi_out_staged(g, rb, p0 + 32 * qtr, lane, q0 + c0 + 32, sbias, stg);
                else epi_chunk(g, rb, row, q0 + c0 + 32, sbias);
                if (c0 + 64 < cb + NCOL) tmem_wait32(ra);
            }
            // this warp's reads of accumulator b are complete: release it to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty(b));
        }
        // the stage must outlive the bulk stores that read it
        if ((tstore || ostore) && lane == 0) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(S::TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------------------------ small kernels

struct InMap {
    float lo[kIn], scale[kIn];   // x' = (x - lo) * scale - 1, scale = 2 / (hi - lo)
};

// raw descriptors [n][6] -> BF16 [npad][64] (zero padded) and, when asked, its transpose
__global__ void k_pack_input(const float *x, int n, int npad, InMap mp, bf16 *a0, bf16 *a0t)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)npad * kK1) return;
    const int r = (int)(e / kK1), k = (int)(e % kK1);
    float v = 0.f;
    if (r < n && k < kIn) v = (x[(long)r * kIn + k] - mp.lo[k]) * mp.scale[k] - 1.f;
    const bf16 b = __float2bfloat16_rn(v);
    a0[e] = b;
    if (a0t) a0t[(long)k * npad + r] = b;
}

// loss partial sums and dL/dy = 2 (y - t) / (B 512) as BF16, row-major and transposed, through
// a 32 x 32 shared-memory tile; block (32, 8), grid (512 / 32, B / 32)
__global__ void k_mse(const float *y, const float *t, int B, float scale, bf16 *dz, bf16 *dzt,
                      double *partial)
{
    __shared__ float tile[32][33];
    __shared__ double red[8];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    double acc = 0.0;
    for (int rr = threadIdx.y; rr < 32; rr += 8) {
        const long e = (long)(r0 + rr) * kOut + c0 + threadIdx.x;
        const float d = y[e] - t[e];
        acc += (double)d * (double)d;
        const float gv = scale * d;
        dz[e] = __float2bfloat16_rn(gv);
        tile[rr][threadIdx.x] = gv;
    }
    __syncthreads();
    for (int cc = threadIdx.y; cc < 32; cc += 8)
        dzt[(long)(c0 + cc) * B + r0 + threadIdx.x] = __float2bfloat16_rn(tile[threadIdx.x][cc]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) red[threadIdx.y] = acc;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// fixed-order sum of the loss partials
__global__ void k_loss_final(const double *partial, int n, double inv, double *loss)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *loss = t * inv;
    }
}

// bias gradient: db[n] = sum_b dz^T[n][b]; one warp per row, fixed order
__global__ void k_rowsum(const bf16 *dzt, int B, int N, float *db)
{
    const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (n >= N) return;
    float s = 0.f;
    for (int b = lane; b < B; b += 32) s += __bfloat162float(dzt[(long)n * B + b]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[n] = s;
}

// Adam with bias correction on the flat FP32 parameters.  The step number k = *kstep + 1 and
// the learning rate (lr_sched[*pos] when a schedule is given, else lr) come from device
// memory, so a captured step replays correctly; k_advance moves both counters afterwards.
struct AdamArgs {
    float *p, *m, *v;
    const float *g;
    long n;
    float lr, b1, b2, eps;
    const long long *kstep;
    const float *lr_sched;
    const int *pos;
};

__global__ void k_adam(AdamArgs a)
{
    const double k = (double)(*a.kstep + 1);
    const float c1 = (float)(1.0 - pow((double)a.b1, k));
    const float c2 = (float)(1.0 - pow((double)a.b2, k));
    const float lr = a.lr_sched ? a.lr_sched[*a.pos] : a.lr;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (long)gridDim.x * blockDim.x) {
        const float gi = a.g[i];
        const float mi = a.b1 * a.m[i] + (1.f - a.b1) * gi;
        const float vi = a.b2 * a.v[i] + (1.f - a.b2) * gi * gi;
        a.m[i] = mi;
        a.v[i] = vi;
        a.p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + a.eps);
    }
}

__global__ void k_advance(long long *kstep, int *pos)
{
    *kstep += 1;
    if (pos) *pos += 1;
}

// training batch of step *pos: rows idx[*pos * B + r] of x [n][6] and t [n][512]
__global__ void k_gather(const float *x, const float *t, const int32_t *idx, const int *pos, int B,
                         int n, float *xin, float *tin, int *status)
{
    const int r = blockIdx.x;
    const long row = idx[(long)(*pos) * B + r];
    if (row < 0 || row >= n) {
        if (threadIdx.x == 0) atomicOr(status, 4);
        return;
    }
    for (int c = threadIdx.x; c < kOut; c += blockDim.x) tin[(long)r * kOut + c] = t[row * kOut + c];
    if (threadIdx.x < kIn) xin[(long)r * kIn + threadIdx.x] = x[row * kIn + threadIdx.x];
}

// FP32 master weights -> BF16 stack [5 * 512][512] (layer l at rows l * 512, K-padded) and the
// transposed stack (layer l >= 1: rows l * 512 + k hold column k of W_l)
__global__ void k_publish(const float *p, bf16 *w, bf16 *wt)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long per = (long)kWidth * kWidth;
    if (e >= kLayers * per) return;
    const int l = (int)(e / per);
    const int n = (int)((e % per) / kWidth), k = (int)(e % kWidth);
    const int in = layer_in(l);
    if (k >= in) return;
    const bf16 b = __float2bfloat16_rn(p[w_off(l) + (long)n * in + k]);
    w[((long)l * kWidth + n) * kWidth + k] = b;
    if (l > 0) wt[((long)l * kWidth + k) * kWidth + n] = b;
}

// Ensemble mean and disagreement: y_m = Y + m * stride, rows [npad][512] laid out as
// [Re S11 | Im S11 | Re S21 | Im S21] x 128 frequencies; one warp per query row.
__global__ void k_ensemble(const float *Y, long stride, int E, int n, float *mean, float *est)
{
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= n) return;
    float dmax = 0.f;
    for (int j = lane; j < 256; j += 32) {
        const int e = j >> 7, f = j & 127;
        const long ire = (long)r * kOut + e * 256 + f, iim = ire + 128;
        float mr = 0.f, mi = 0.f;
        for (int m = 0; m < E; ++m) {
            mr += Y[m * stride + ire];
            mi += Y[m * stride + iim];
        }
        mr /= (float)E;
        mi /= (float)E;
        for (int m = 0; m < E; ++m) {
            const float dr = Y[m * stride + ire] - mr, di = Y[m * stride + iim] - mi;
            dmax = fmaxf(dmax, sqrtf(dr * dr + di * di));
        }
        mean[ire] = mr;
        mean[iim] = mi;
    }
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if (lane == 0 && est) est[r] = dmax;
}

__global__ void k_gate(const float *est, int n, float scale, float thr, int32_t *flags, int *count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int f = 0;
    if (i < n) {
        f = scale * est[i] > thr;
        flags[i] = f;
    }
    const unsigned b = __ballot_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(count, __popc(b));
}

}  // namespace mlp
}  // namespace yf

// ------------------------------------------------------------------ host side

using namespace yf;
using namespace yf::mlp;

struct yf_mlp {
    int E = 0, B = 0, NQ = 0, nq_max = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    InMap in;
    double lr = 1e-3, b1 = 0.9, b2 = 0.999, eps = 1e-8;
    long long *kstep = nullptr;   // per member Adam step count (device)
    int *pos = nullptr;           // step index inside the current yf_mlp_fit call (device)
    // captured training step per member, valid for the pointers it was captured with
    std::vector<cudaGraphExec_t> fit_graph;
    struct FitKey { const void *x, *t, *idx, *lr; int n; };
    std::vector<FitKey> fit_key;
    // per member
    std::vector<float *> master, mom, vel, grad;
    std::vector<bf16 *> wst, wtst;
    std::vector<CUtensorMap> mW, mWT;
    // training buffers
    float *xin = nullptr, *tin = nullptr, *y = nullptr, *z[kLayers - 1] = {};
    bf16 *a0 = nullptr, *a0t = nullptr, *act[kLayers - 1] = {}, *actt[kLayers - 1] = {};
    bf16 *dz[kLayers] = {}, *dzt[kLayers] = {};
    double *partial = nullptr, *loss = nullptr;
    CUtensorMap mA0, mA0T, mAct[kLayers - 1], mActT[kLayers - 1], mDz[kLayers], mDzT[kLayers];
    // query buffers
    float *qx = nullptr, *qY = nullptr, *qmean = nullptr, *qest = nullptr;
    bf16 *qa0 = nullptr, *qact[2] = {};
    CUtensorMap mQA0, mQAct[2], mQActSt[2];   // mQActSt: 32 x 32 boxes for the bulk stores
    CUtensorMap mQYSt;                        // qY of all members, 16 x 32 FP32 boxes
    int *status = nullptr, *count = nullptr;
    std::vector<void *> allocs;
};

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D BF16 map over a row-major [rows][cols] matrix, box 64 columns x box_rows rows, 128-byte
// swizzle (the layout the tcgen05 descriptors above expect)
yf_status map2d(CUtensorMap *m, const void *base, long rows, long cols, int box_rows)
{
    auto enc = encoder();
    if (!enc) return fail(YF_E_CUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t str[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t one[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dim, str, box, one,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(YF_E_CUDA, "encoding an MLP tensor map failed (%d)", (int)r);
    return YF_OK;
}

// 2-D map for the bulk stores of the inference epilogues: boxes of 32 rows of 64 bytes (32 BF16
// or 16 FP32 columns), 64-byte swizzle (the stage layout epi_hidden_tma and epi_out_tma write)
yf_status map2d_store(CUtensorMap *m, const void *base, long rows, long cols,
                      CUtensorMapDataType type = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, int box_cols = 32)
{
    auto enc = encoder();
    if (!enc) return fail(YF_E_CUDA, "cuTensorMapEncodeTiled is not available");
    const int esz = type == CU_TENSOR_MAP_DATA_TYPE_FLOAT32 ? 4 : 2;
    const cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t str[1] = {(cuuint64_t)cols * esz};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, 32};   // rows of 64 bytes
    const cuuint32_t one[2] = {1, 1};
    CUresult r = enc(m, type, 2, const_cast<void *>(base), dim, str, box, one,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(YF_E_CUDA, "encoding an MLP store map failed (%d)", (int)r);
    return YF_OK;
}

template <typename T>
yf_status dalloc(yf_mlp *m, T **p, size_t count)
{
    void *v = nullptr;
    if (cudaMalloc(&v, count * sizeof(T) + 16) != cudaSuccess) {
        cudaGetLastError();
        return fail(YF_E_OOM, "yf_mlp: device allocation of %zu bytes failed", count * sizeof(T));
    }
    m->allocs.push_back(v);
    *p = (T *)v;
    YF_CUDA_TRY(cudaMemset(v, 0, count * sizeof(T) + 16));
    return YF_OK;
}

template <int NT>
cudaError_t prepare_persist()
{
    return cudaFuncSetAttribute(k_mlp_gemm_persist<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                PersistSmem<NT>::BYTES);
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 148;
    }
    return n;
}

template <int NT, int ST>
cudaError_t prepare_gemm()
{
    return cudaFuncSetAttribute(k_mlp_gemm<NT, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                GemmSmem<NT, ST>::BYTES);
}

template <int NT, int ST>
cudaError_t launch_gemm_t(const CUtensorMap &a, const CUtensorMap &b, const GemmArgs &g, cudaStream_t s)
{
    dim3 grid(g.P / kBM, g.Q / NT);
    k_mlp_gemm<NT, ST><<<grid, kThreads, GemmSmem<NT, ST>::BYTES, s>>>(a, b, g);
    return cudaGetLastError();
}

// Large grids (at least two tiles per SM) take 2 stages: 96 KB of shared memory and 256 TMEM
// columns per CTA let two CTAs share an SM, so one's epilogue overlaps the other's MMAs.
// Small grids (the training GEMMs) keep 4 stages for a deeper copy pipeline.
// c: store map of the output for the hidden-layer inference epilogue (with g.tma_store), else null
cudaError_t launch_gemm(const CUtensorMap &a, const CUtensorMap &b, const GemmArgs &g, cudaStream_t s,
                        const CUtensorMap *c = nullptr)
{
    if (g.Q % 256 == 0) {
        const long tiles = (long)(g.P / kBM) * (g.Q / 256);
        if (tiles >= 2 * sm_count()) {
            // persistent: one CTA per SM (its shared memory admits no second one)
            k_mlp_gemm_persist<256><<<sm_count(), kThreads, PersistSmem<256>::BYTES, s>>>(a, b, c ? *c : a, g);
            return cudaGetLastError();
        }
        return launch_gemm_t<256, 4>(a, b, g, s);
    }
    return launch_gemm_t<64, 4>(a, b, g, s);
}

GemmArgs args(yf_mlp *m, int P, int Q, int R, int mode)
{
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.P = P; g.Q = Q; g.R = R; g.mode = mode; g.qvalid = Q; g.status = m->status;
    return g;
}

yf_status check_status(yf_mlp *m)
{
    int st = 0;
    YF_CUDA_TRY(cudaMemcpyAsync(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    YF_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (st) {
        YF_CUDA_TRY(cudaMemsetAsync(m->status, 0, sizeof(int), m->stream));
        if (st & 2) return fail(YF_E_TIMEOUT, "yf_mlp: a tensor-core pipeline wait gave up (status %d)", st);
        return fail(YF_E_INVALID, "yf_mlp_fit: a training row index was outside [0, n)");
    }
    return YF_OK;
}

// forward + backward of one member on the staged training batch; gradients land in grad[member]
yf_status train_pass(yf_mlp *m, int mem)
{
    const int B = m->B;
    cudaStream_t s = m->stream;
    k_pack_input<<<(B * kK1 + 255) / 256, 256, 0, s>>>(m->xin, B, B, m->in, m->a0, m->a0t);
    YF_CUDA_TRY(cudaGetLastError());
    const float *P = m->master[mem];
    for (int l = 0; l < kLayers; ++l) {
        const bool last = l == kLayers - 1;
        GemmArgs g = args(m, B, kWidth, l == 0 ? kK1 : kWidth, last ? MODE_OUT : MODE_HIDDEN);
        g.b_row0 = l * kWidth;
        g.bias = P + b_off(l);
        if (last) {
            g.out_f32 = m->y; g.ld_f32 = kOut;
        } else {
            g.out_f32 = m->z[l]; g.ld_f32 = kWidth;
            g.out_bf = m->act[l]; g.ld_bf = kWidth;
            g.out_t = m->actt[l]; g.ld_t = B;
        }
        YF_CUDA_TRY(launch_gemm(l == 0 ? m->mA0 : m->mAct[l - 1], m->mW[mem], g, s));
    }
    k_mse<<<dim3(kOut / 32, B / 32), dim3(32, 8), 0, s>>>(m->y, m->tin, B, 2.f / ((float)B * kOut),
                                                         m->dz[kLayers - 1], m->dzt[kLayers - 1], m->partial);
    YF_CUDA_TRY(cudaGetLastError());
    k_loss_final<<<1, 256, 0, s>>>(m->partial, (kOut / 32) * (B / 32), 1.0 / ((double)B * kOut), m->loss);
    YF_CUDA_TRY(cudaGetLastError());
    float *G = m->grad[mem];
    for (int l = kLayers - 1; l >= 0; --l) {
        const int in = layer_in(l);
        GemmArgs w = args(m, kWidth, l == 0 ? kK1 : kWidth, B, MODE_WGRAD);
        w.out_f32 = G + w_off(l); w.ld_f32 = in; w.qvalid = in;
        YF_CUDA_TRY(launch_gemm(m->mDzT[l], l == 0 ? m->mA0T : m->mActT[l - 1], w, s));
        k_rowsum<<<kWidth / 8, 256, 0, s>>>(m->dzt[l], B, kWidth, G + b_off(l));
        YF_CUDA_TRY(cudaGetLastError());
        if (l > 0) {
            GemmArgs d = args(m, B, kWidth, kWidth, MODE_DGRAD);
            d.b_row0 = l * kWidth;
            d.zin = m->z[l - 1]; d.ld_z = kWidth;
            d.out_bf = m->dz[l - 1]; d.ld_bf = kWidth;
            d.out_t = m->dzt[l - 1]; d.ld_t = B;
            YF_CUDA_TRY(launch_gemm(m->mDz[l], m->mWT[mem], d, s));
        }
    }
    return YF_OK;
}

yf_status stage_batch(yf_mlp *m, const float *x, const float *t, yf_mem where)
{
    const cudaMemcpyKind k = where == YF_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    YF_CUDA_TRY(cudaMemcpyAsync(m->xin, x, (size_t)m->B * kIn * sizeof(float), k, m->stream));
    YF_CUDA_TRY(cudaMemcpyAsync(m->tin, t, (size_t)m->B * kOut * sizeof(float), k, m->stream));
    return YF_OK;
}

yf_status publish(yf_mlp *m, int mem)
{
    const long n = (long)kLayers * kWidth * kWidth;
    k_publish<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->master[mem], m->wst[mem], m->wtst[mem]);
    YF_CUDA_TRY(cudaGetLastError());
    return YF_OK;
}

cudaError_t adam_step(yf_mlp *m, int mem, const float *lr_sched)
{
    AdamArgs a;
    a.p = m->master[mem]; a.m = m->mom[mem]; a.v = m->vel[mem]; a.g = m->grad[mem];
    a.n = kParams;
    a.lr = (float)m->lr; a.b1 = (float)m->b1; a.b2 = (float)m->b2; a.eps = (float)m->eps;
    a.kstep = m->kstep + mem;
    a.lr_sched = lr_sched;
    a.pos = m->pos;
    k_adam<<<148 * 8, 256, 0, m->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_advance<<<1, 1, 0, m->stream>>>(m->kstep + mem, lr_sched ? m->pos : nullptr);
    return cudaGetLastError();
}

bool bad_member(yf_mlp *m, int mem) { return !m || mem < 0 || mem >= m->E; }

}  // namespace

extern "C" {

yf_status yf_mlp_create(int members, int train_batch, int max_query, const double *in_lo,
                        const double *in_hi, void *stream, yf_mlp **out)
{
    if (!out || !in_lo || !in_hi) return fail(YF_E_INVALID, "yf_mlp_create: NULL argument");
    *out = nullptr;
    if (members < 1 || members > 8) return fail(YF_E_INVALID, "yf_mlp_create: members must be 1..8");
    if (train_batch < kBM || train_batch % kBM) return fail(YF_E_INVALID, "yf_mlp_create: train_batch must be a positive multiple of 128");
    if (max_query < 1) return fail(YF_E_INVALID, "yf_mlp_create: max_query must be >= 1");
    for (int k = 0; k < kIn; ++k)
        if (!(in_hi[k] > in_lo[k])) return fail(YF_E_INVALID, "yf_mlp_create: in_hi must exceed in_lo");
    if (!encoder()) return fail(YF_E_CUDA, "cuTensorMapEncodeTiled is not available");
    yf_mlp *m = new yf_mlp;
    m->E = members;
    m->B = train_batch;
    m->nq_max = max_query;
    m->NQ = (max_query + kBM - 1) / kBM * kBM;
    for (int k = 0; k < kIn; ++k) {
        m->in.lo[k] = (float)in_lo[k];
        m->in.scale[k] = (float)(2.0 / (in_hi[k] - in_lo[k]));
    }
    auto bail = [&](yf_status st) {
        yf_mlp_destroy(m);
        return st;
    };
    if (stream) {
        m->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "cudaStreamCreateWithFlags"));
        m->own_stream = true;
    }
    if (prepare_gemm<256, 4>() != cudaSuccess || prepare_gemm<64, 4>() != cudaSuccess ||
        prepare_persist<256>() != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaFuncSetAttribute(k_mlp_gemm)"));
    yf_status st;
#define TRY(x)                                \
    do {                                      \
        if ((st = (x)) != YF_OK) return bail(st); \
    } while (0)
    const long stackn = (long)kLayers * kWidth * kWidth;
    m->fit_graph.assign(members, nullptr);
    m->fit_key.assign(members, yf_mlp::FitKey{nullptr, nullptr, nullptr, nullptr, 0});
    m->master.resize(members); m->mom.resize(members); m->vel.resize(members); m->grad.resize(members);
    m->wst.resize(members); m->wtst.resize(members); m->mW.resize(members); m->mWT.resize(members);
    for (int e = 0; e < members; ++e) {
        TRY(dalloc(m, &m->master[e], kParams));
        TRY(dalloc(m, &m->mom[e], kParams));
        TRY(dalloc(m, &m->vel[e], kParams));
        TRY(dalloc(m, &m->grad[e], kParams));
        TRY(dalloc(m, &m->wst[e], stackn));
        TRY(dalloc(m, &m->wtst[e], stackn));
        TRY(map2d(&m->mW[e], m->wst[e], (long)kLayers * kWidth, kWidth, 256));
        TRY(map2d(&m->mWT[e], m->wtst[e], (long)kLayers * kWidth, kWidth, 256));
    }
    const int B = train_batch;
    TRY(dalloc(m, &m->xin, (size_t)B * kIn));
    TRY(dalloc(m, &m->tin, (size_t)B * kOut));
    TRY(dalloc(m, &m->y, (size_t)B * kOut));
    TRY(dalloc(m, &m->a0, (size_t)B * kK1));
    TRY(dalloc(m, &m->a0t, (size_t)B * kK1));
    TRY(map2d(&m->mA0, m->a0, B, kK1, kBM));
    TRY(map2d(&m->mA0T, m->a0t, kK1, B, 64));
    for (int l = 0; l < kLayers - 1; ++l) {
        TRY(dalloc(m, &m->z[l], (size_t)B * kWidth));
        TRY(dalloc(m, &m->act[l], (size_t)B * kWidth));
        TRY(dalloc(m, &m->actt[l], (size_t)B * kWidth));
        TRY(map2d(&m->mAct[l], m->act[l], B, kWidth, kBM));
        TRY(map2d(&m->mActT[l], m->actt[l], kWidth, B, 256));
    }
    for (int l = 0; l < kLayers; ++l) {
        TRY(dalloc(m, &m->dz[l], (size_t)B * kWidth));
        TRY(dalloc(m, &m->dzt[l], (size_t)B * kWidth));
        TRY(map2d(&m->mDz[l], m->dz[l], B, kWidth, kBM));
        TRY(map2d(&m->mDzT[l], m->dzt[l], kWidth, B, kBM));
    }
    TRY(dalloc(m, &m->partial, (size_t)(kOut / 32) * (B / 32)));
    TRY(dalloc(m, &m->loss, 1));
    const int NQ = m->NQ;
    TRY(dalloc(m, &m->qx, (size_t)NQ * kIn));
    TRY(dalloc(m, &m->qa0, (size_t)NQ * kK1));
    TRY(map2d(&m->mQA0, m->qa0, NQ, kK1, kBM));
    for (int b = 0; b < 2; ++b) {
        TRY(dalloc(m, &m->qact[b], (size_t)NQ * kWidth));
        TRY(map2d(&m->mQAct[b], m->qact[b], NQ, kWidth, kBM));
        TRY(map2d_store(&m->mQActSt[b], m->qact[b], NQ, kWidth));
    }
    TRY(dalloc(m, &m->qY, (size_t)members * NQ * kOut));
    TRY(map2d_store(&m->mQYSt, m->qY, (long)members * NQ, kOut, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 16));
    TRY(dalloc(m, &m->qmean, (size_t)NQ * kOut));
    TRY(dalloc(m, &m->qest, (size_t)NQ));
    TRY(dalloc(m, &m->status, 1));
    TRY(dalloc(m, &m->count, 1));
    TRY(dalloc(m, &m->kstep, (size_t)members));
    TRY(dalloc(m, &m->pos, 1));
#undef TRY
    *out = m;
    return YF_OK;
}

yf_status yf_mlp_destroy(yf_mlp *m)
{
    if (!m) return YF_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (cudaGraphExec_t g : m->fit_graph)
        if (g) cudaGraphExecDestroy(g);
    for (void *p : m->allocs) cudaFree(p);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return YF_OK;
}

yf_status yf_mlp_set_params(yf_mlp *m, int member, const double *params)
{
    if (bad_member(m, member) || !params) return fail(YF_E_INVALID, "yf_mlp_set_params: bad argument");
    std::vector<float> f(kParams);
    for (long i = 0; i < kParams; ++i) f[i] = (float)params[i];
    YF_CUDA_TRY(cudaMemcpyAsync(m->master[member], f.data(), kParams * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    YF_CUDA_TRY(cudaMemsetAsync(m->mom[member], 0, kParams * sizeof(float), m->stream));
    YF_CUDA_TRY(cudaMemsetAsync(m->vel[member], 0, kParams * sizeof(float), m->stream));
    YF_CUDA_TRY(cudaMemsetAsync(m->kstep + member, 0, sizeof(long long), m->stream));
    yf_status st = publish(m, member);
    if (st != YF_OK) return st;
    YF_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return YF_OK;
}

yf_status yf_mlp_get_params(yf_mlp *m, int member, double *params)
{
    if (bad_member(m, member) || !params) return fail(YF_E_INVALID, "yf_mlp_get_params: bad argument");
    std::vector<float> f(kParams);
    YF_CUDA_TRY(cudaMemcpyAsync(f.data(), m->master[member], kParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    YF_CUDA_TRY(cudaStreamSynchronize(m->stream));
    for (long i = 0; i < kParams; ++i) params[i] = f[i];
    return YF_OK;
}

yf_status yf_mlp_set_adam(yf_mlp *m, double lr, double beta1, double beta2, double eps)
{
    if (!m || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return fail(YF_E_INVALID, "yf_mlp_set_adam: bad hyper-parameters");
    m->lr = lr; m->b1 = beta1; m->b2 = beta2; m->eps = eps;
    return YF_OK;
}

yf_status yf_mlp_grads(yf_mlp *m, int member, const float *x, const float *t, yf_mem where,
                       double *loss, double *grads)
{
    if (bad_member(m, member) || !x || !t) return fail(YF_E_INVALID, "yf_mlp_grads: bad argument");
    yf_status st = stage_batch(m, x, t, where);
    if (st != YF_OK) return st;
    if ((st = train_pass(m, member)) != YF_OK) return st;
    if ((st = check_status(m)) != YF_OK) return st;
    if (loss) YF_CUDA_TRY(cudaMemcpy(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost));
    if (grads) {
        std::vector<float> f(kParams);
        YF_CUDA_TRY(cudaMemcpy(f.data(), m->grad[member], kParams * sizeof(float), cudaMemcpyDeviceToHost));
        for (long i = 0; i < kParams; ++i) grads[i] = f[i];
    }
    return YF_OK;
}

yf_status yf_mlp_train_step(yf_mlp *m, int member, const float *x, const float *t, yf_mem where,
                            double *loss)
{
    if (bad_member(m, member) || !x || !t) return fail(YF_E_INVALID, "yf_mlp_train_step: bad argument");
    yf_status st = stage_batch(m, x, t, where);
    if (st != YF_OK) return st;
    if ((st = train_pass(m, member)) != YF_OK) return st;
    YF_CUDA_TRY(adam_step(m, member, nullptr));
    if ((st = publish(m, member)) != YF_OK) return st;
    if (loss) {
        if ((st = check_status(m)) != YF_OK) return st;
        YF_CUDA_TRY(cudaMemcpy(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost));
    }
    return YF_OK;
}

yf_status yf_mlp_fit(yf_mlp *m, int member, const float *x, const float *t, int n,
                     const int32_t *idx, const float *lr, long steps)
{
    if (bad_member(m, member) || !x || !t || !idx || !lr || n < 1 || steps < 0)
        return fail(YF_E_INVALID, "yf_mlp_fit: bad argument");
    if (steps == 0) return YF_OK;
    yf_mlp::FitKey key{x, t, idx, lr, n};
    yf_mlp::FitKey &old = m->fit_key[member];
    const bool same = old.x == key.x && old.t == key.t && old.idx == key.idx && old.lr == key.lr &&
                      old.n == key.n;
    if (!m->fit_graph[member] || !same) {
        if (m->fit_graph[member]) {
            cudaGraphExecDestroy(m->fit_graph[member]);
            m->fit_graph[member] = nullptr;
        }
        cudaGraph_t graph = nullptr;
        YF_CUDA_TRY(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
        k_gather<<<m->B, 128, 0, m->stream>>>(x, t, idx, m->pos, m->B, n, m->xin, m->tin, m->status);
        yf_status st = train_pass(m, member);
        cudaError_t e = st == YF_OK ? adam_step(m, member, lr) : cudaSuccess;
        if (e == cudaSuccess && st == YF_OK) st = publish(m, member);
        cudaError_t ec = cudaStreamEndCapture(m->stream, &graph);
        if (st != YF_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e != cudaSuccess ? e : ec, "capturing the training step");
        }
        e = cudaGraphInstantiate(&m->fit_graph[member], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(training step)");
        old = key;
    }
    YF_CUDA_TRY(cudaMemsetAsync(m->pos, 0, sizeof(int), m->stream));
    for (long s = 0; s < steps; ++s) YF_CUDA_TRY(cudaGraphLaunch(m->fit_graph[member], m->stream));
    return YF_OK;
}

yf_status yf_mlp_sync(yf_mlp *m, double *loss)
{
    if (!m) return fail(YF_E_INVALID, "yf_mlp_sync: NULL handle");
    yf_status st = check_status(m);
    if (st != YF_OK) return st;
    if (loss) YF_CUDA_TRY(cudaMemcpy(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost));
    return YF_OK;
}

yf_status yf_mlp_query(yf_mlp *m, const float *x, int n, yf_mem where, float *y, float *est,
                       yf_mem out_where)
{
    if (!m || !x || !y || n < 1 || n > m->nq_max) return fail(YF_E_INVALID, "yf_mlp_query: bad argument");
    cudaStream_t s = m->stream;
    const int np = (n + kBM - 1) / kBM * kBM;
    YF_CUDA_TRY(cudaMemcpyAsync(m->qx, x, (size_t)n * kIn * sizeof(float),
                                where == YF_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    k_pack_input<<<(unsigned)(((long)np * kK1 + 255) / 256), 256, 0, s>>>(m->qx, n, np, m->in, m->qa0, nullptr);
    YF_CUDA_TRY(cudaGetLastError());
    const long ystride = (long)m->NQ * kOut;
    for (int e = 0; e < m->E; ++e) {
        for (int l = 0; l < kLayers; ++l) {
            const bool last = l == kLayers - 1;
            GemmArgs g = args(m, np, kWidth, l == 0 ? kK1 : kWidth, last ? MODE_OUT : MODE_HIDDEN);
            g.b_row0 = l * kWidth;
            g.bias = m->master[e] + b_off(l);
            if (last) {
                g.out_f32 = m->qY + e * ystride; g.ld_f32 = kOut;
                g.tma_store = 1;
                g.out_row0 = e * m->NQ;
            } else {
                g.out_bf = m->qact[l & 1]; g.ld_bf = kWidth;
                g.tma_store = 1;
            }
            const CUtensorMap &a = l == 0 ? m->mQA0 : m->mQAct[(l - 1) & 1];
            YF_CUDA_TRY(launch_gemm(a, m->mW[e], g, s, last ? &m->mQYSt : &m->mQActSt[l & 1]));
        }
    }
    if (out_where == YF_DEVICE) {
        // device outputs: the ensemble pass writes them in place (no staging copy)
        k_ensemble<<<(n + 7) / 8, 256, 0, s>>>(m->qY, ystride, m->E, n, y, est);
        YF_CUDA_TRY(cudaGetLastError());
        return YF_OK;
    }
    k_ensemble<<<(n + 7) / 8, 256, 0, s>>>(m->qY, ystride, m->E, n, m->qmean, m->qest);
    YF_CUDA_TRY(cudaGetLastError());
    YF_CUDA_TRY(cudaMemcpyAsync(y, m->qmean, (size_t)n * kOut * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (est) YF_CUDA_TRY(cudaMemcpyAsync(est, m->qest, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s));
    return check_status(m);
}

yf_status yf_mlp_gate(yf_mlp *m, const float *est, int n, double scale, double threshold,
                      yf_mem where, int32_t *flags, int *nflagged)
{
    if (!m || !est || !flags || n < 1) return fail(YF_E_INVALID, "yf_mlp_gate: bad argument");
    cudaStream_t s = m->stream;
    const float *e_dev = est;
    int32_t *f_dev = flags;
    std::vector<int32_t> host_flags;
    if (where == YF_HOST) {
        if (n > m->nq_max) return fail(YF_E_INVALID, "yf_mlp_gate: host arrays are limited to max_query entries");
        YF_CUDA_TRY(cudaMemcpyAsync(m->qest, est, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, s));
        e_dev = m->qest;
        f_dev = (int32_t *)m->qY;   // scratch: the flags fit in the output buffer
    }
    YF_CUDA_TRY(cudaMemsetAsync(m->count, 0, sizeof(int), s));
    k_gate<<<(n + 255) / 256, 256, 0, s>>>(e_dev, n, (float)scale, (float)threshold, f_dev, m->count);
    YF_CUDA_TRY(cudaGetLastError());
    if (where == YF_HOST) YF_CUDA_TRY(cudaMemcpyAsync(flags, f_dev, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (nflagged) {
        YF_CUDA_TRY(cudaMemcpyAsync(nflagged, m->count, sizeof(int), cudaMemcpyDeviceToHost, s));
        YF_CUDA_TRY(cudaStreamSynchronize(s));
    } else if (where == YF_HOST) {
        YF_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return YF_OK;
}

yf_status yf_mlp_query_stats(yf_mlp *m, int *launches, double *gemm_flops)
{
    if (!m) return fail(YF_E_INVALID, "yf_mlp_query_stats: NULL handle");
    if (launches) *launches = 2 + m->E * kLayers;
    // algorithmic: the layer-1 K of 6, not the padded 64 the tensor cores run
    if (gemm_flops) *gemm_flops = 2.0 * m->E * ((double)kIn * kWidth + 3.0 * kWidth * kWidth + (double)kWidth * kOut);
    return YF_OK;
}

}  // extern "C"
