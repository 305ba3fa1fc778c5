// tc.cuh -- the pieces of the sm_103a fifth-generation tensor core (tcgen05)
// the stage products of the large shapes use: tensor-memory (TMEM)
// allocation, shared-memory matrix descriptors, instruction descriptors of
// kind::tf32 and kind::f16 (BF16 operands) with an FP32 accumulator in TMEM,
// completion through an mbarrier, and TMEM -> register loads.  Written from the
// PTX ISA's tcgen05 chapter:
//
//  * Operands live in shared memory in the canonical K-major layout without
//    swizzling: "core matrices" of 8 rows x 16 bytes (8 x 4 TF32 or 8 x 8 BF16
//    values, 128 contiguous bytes); the descriptor gives the byte distance
//    between core matrices adjacent along K (leading byte offset) and between
//    8-row groups (stride byte offset).  Element (r, k) of a 32-bit tile sits at
//    (r / 8) * sbo + (k / 4) * lbo + (r % 8) * 16 + (k % 4) * 4 bytes.
//  * D[m][n] = sum_k A[m][k] B[n][k]: both operands K-major, M = 128 rows of A,
//    N rows of B (a multiple of 16, at most 256), K = 8 (TF32) or 16 (BF16) per
//    instruction.
//  * The accumulator of an M = 128 MMA holds row m in TMEM lane m, column n in
//    TMEM column (base + n); warp w of a four-warp team reads lanes 32w..32w+31
//    (32x32b shape: thread t of the warp gets lane 32w + t).
//  * One thread issues the MMAs and commits them to an mbarrier; every thread
//    waits on the mbarrier's phase, with an iteration limit.
//
// Accuracy: a TF32 operand keeps 10 fraction bits, a BF16 operand 7.  The
// products that need FP32 accuracy split each operand into TF32 hi + lo or
// BF16 hi + mid + lo and keep the terms of each magnitude in an accumulator of
// their own (small terms added into a large accumulator lose bits to its
// alignment); tree.cuh: tc_stage_products and tc_stage_products_bf16.
#pragma once
#include <stdint.h>

#include "warp.cuh"

#ifdef __CUDACC__
#define MHE_TC_HD __host__ __device__
#else
#define MHE_TC_HD
#endif

namespace mhe {
MHE_TEAM_NS_BEGIN
namespace tc {

// x rounded to the nearest TF32 value (ties away from zero) in integer
// arithmetic on the bit pattern: the 13 low fraction bits are rounded off.
MHE_DEV float tf32_hi(float x)
{
    const unsigned b = __float_as_uint(x);
    return __uint_as_float((b + 0x1000u) & 0xFFFFE000u);
}

// byte offset of element (r, k) in a canonical K-major tile of 32-bit elements
MHE_TC_HD constexpr int kmaj_off(int r, int k, int lbo, int sbo)
{
    return (r / 8) * sbo + (k / 4) * lbo + (r % 8) * 16 + (k % 4) * 4;
}

// the same for 16-bit elements (a core matrix row holds 8 of them)
MHE_TC_HD constexpr int kmaj_off16(int r, int k, int lbo, int sbo)
{
    return (r / 8) * sbo + (k / 8) * lbo + (r % 8) * 16 + (k % 8) * 2;
}

// x rounded to the nearest BF16 value (ties to even), as its 16 bits and as a
// float; integer arithmetic on the bit pattern (finite x)
MHE_DEV unsigned short bf16_bits(float x)
{
    const unsigned b = __float_as_uint(x);
    return (unsigned short)((b + 0x7FFFu + ((b >> 16) & 1u)) >> 16);
}
MHE_DEV float bf16_val(unsigned short h) { return __uint_as_float((unsigned)h << 16); }

// instruction descriptor: kind::f16 with BF16 A and B (format 1), FP32 accumulator,
// both K-major, N / 8 in bits 17-22, M / 16 in bits 24-28
MHE_TC_HD constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// instruction descriptor: kind::tf32, dense, FP32 accumulator (D format 1),
// A and B TF32 (format 2), both K-major, no negation, N / 8 in bits 17-22,
// M / 16 in bits 24-28
MHE_TC_HD constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

#ifndef MHE_TC_EMULATED

MHE_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading and stride byte
// offsets (each encoded >> 4 in 14 bits), bits 46-48 = 0b001, base offset 0,
// relative leading offset, no swizzle
MHE_DEV uint64_t sdesc(const void* p, uint32_t lbo, uint32_t sbo)
{
    const uint32_t a = smem_u32(p);
    uint64_t d = (uint64_t)((a & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// TMEM allocation of ncols columns (a power of two >= 32) by one whole warp;
// the TMEM address is written to *slot (shared memory)
MHE_DEV void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

MHE_DEV void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (+)= A B^T, one instruction of K = 8
MHE_DEV void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// D (+)= A B^T with BF16 operands, one instruction of K = 16
MHE_DEV void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// the mbarrier at m completes a phase when the MMAs this thread issued so far are done
MHE_DEV void commit(uint64_t* m)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(m))
                 : "memory");
}

MHE_DEV void mbar_init(uint64_t* m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// wait for the phase of the given parity to complete, at most `limit` tries
// (each try suspends the thread for a bounded, system-dependent time)
MHE_DEV bool mbar_wait(uint64_t* m, uint32_t parity, int limit)
{
    const uint32_t a = smem_u32(m);
    for (int i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

MHE_DEV void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
MHE_DEV void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core's (async proxy) reads
MHE_DEV void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive accumulator columns of this thread's TMEM lane (lane = the
// thread's index in its four-warp team; its warp reads its quarter of the
// lanes), load and wait in one statement so no use of the registers can be
// scheduled before the data has arrived
MHE_DEV void tmem_ld16(uint32_t tbase, int /*lane*/, int col, float (&v)[16])
{
    const uint32_t warp = (threadIdx.x >> 5) & 3u;
    const uint32_t ta = tbase + ((warp * 32u) << 16) + (uint32_t)col;
    uint32_t r[16];
    __syncwarp();   // the load is warp-collective
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// two blocks of 16 columns (at col_a and col_b) of this thread's lane, one wait
MHE_DEV void tmem_ld16x2(uint32_t tbase, int /*lane*/, int col_a, int col_b, float (&va)[16], float (&vb)[16])
{
    const uint32_t warp = (threadIdx.x >> 5) & 3u;
    const uint32_t ta = tbase + ((warp * 32u) << 16) + (uint32_t)col_a;
    const uint32_t tb = tbase + ((warp * 32u) << 16) + (uint32_t)col_b;
    uint32_t r[32];
    __syncwarp();
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta), "r"(tb));
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        va[i] = __uint_as_float(r[i]);
        vb[i] = __uint_as_float(r[16 + i]);
    }
}

// tries of an mbarrier wait before a team gives up (each try suspends for a
// bounded time; the MMAs of one stage take microseconds)
constexpr int kWaitLimit = 1 << 20;

// Tries of the product waits when >= 0 (a test setting, default -1: kWaitLimit);
// the wait that frees TMEM after a failed one always takes kWaitLimit.  One copy
// per translation unit: the tensor-core kernels' unit sets its own.
static __device__ int g_wait_override = -1;

// every thread of the team (= the CTA) waits for the phase; true when all saw
// it complete.  Accumulator reads may follow.
MHE_DEV bool team_wait(uint64_t* m, uint32_t parity)
{
    const int lim = g_wait_override >= 0 ? g_wait_override : kWaitLimit;
    const bool ok = mbar_wait(m, parity, lim);
    const bool all = __syncthreads_and(ok) != 0;
    fence_after();
    return all;
}

// every lane runs f (its index in the team), then the tiles it wrote are
// published to the tensor core: proxy fence, tensor fence, one team barrier
template <class F>
MHE_DEV void lanes_publish(F&& f)
{
    f(lane_id());
    fence_smem_to_async();
    fence_before();
    wsync();
}

#endif  // MHE_TC_EMULATED

}  // namespace tc
MHE_TEAM_NS_END
}  // namespace mhe
