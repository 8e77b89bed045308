// tcgen05 / mbarrier helpers and the shared-memory operand layouts used by
// the tensor-core kernels (inline PTX for sm_103a).
//
// A operand: K-major, 128-byte swizzle, [128 rows][64 K] 16-bit elements
// (16 KB per plane); B operand: MN-major, 128-byte swizzle, [64 K][128 N]
// 16-bit elements (two 64-column atoms); accumulators FP32 in TMEM.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace qmc {
constexpr int TC_M = 128, TC_N = 128, TC_K = 64;
constexpr int kTcThreads = 512;   // four threads per walker row
constexpr uint32_t kAPlaneBytes = TC_M * TC_K * 2;     // 16 KB, one output x one split
constexpr uint32_t kBPlaneBytes = TC_K * TC_N * 2;     // 16 KB, one split
constexpr uint32_t kBLbo = 1024;                        // MN-major: next 64-column atom
constexpr uint32_t kBSbo = 2048;                        // MN-major: next group of 8 K rows
constexpr int TC_OUT = 3;                               // C2, C3, C4
constexpr uint32_t kTcSmemFixed = 2 * TC_OUT * kAPlaneBytes + 2 * kBPlaneBytes;   // 128 KB of operands

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor, 128-byte swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;    // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;    // SWIZZLE_128B
    return d;
}

// kind::f16 instruction descriptor: D = F32, A and B both FP16 (format 0) or
// both BF16 (format 1), A K-major, B MN-major, shape M x N.
__host__ __device__ constexpr uint32_t umma_idesc_f16(int M, int N, int bf16)
{
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | (0u << 15) | (1u << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The same with both operand majors given: a_mn / b_mn = 1 for an MN-major
// operand (transpose bits 15 and 16 of the descriptor), 0 for K-major.
__host__ __device__ constexpr uint32_t umma_idesc_f16_major(int M, int N, int bf16, int a_mn, int b_mn)
{
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)a_mn << 15) |
           ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
static_assert(umma_idesc_f16_major(128, 96, 1, 0, 1) == umma_idesc_f16(128, 96, 1), "descriptor fields");

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One test of the mbarrier phase with the given parity (true: that phase has completed).
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    return done != 0;
}

// Bounded wait for the mbarrier phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint64_t limit_ns)
{
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(mbar, parity)) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(mbar) : "memory");
}

// Arrive and add `bytes` to the phase's expected transaction count (the bulk copies that
// complete on this barrier count their bytes down).
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}

// Bulk copy global -> this CTA's shared memory (the TMA's untiled form): both addresses
// 16-byte aligned, bytes a multiple of 16; completion counted in bytes on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

// Bounded wait on a flag that nothing in the kernel sets (the test hook that
// makes a CTA's wait run out, WaitCfg::expire_w); returns false after limit_ns.
__device__ __forceinline__ bool flag_wait(const volatile int *f, uint64_t limit_ns)
{
    const uint64_t t0 = globaltimer();
    while (!*f)
        if (globaltimer() - t0 > limit_ns) return false;
    return true;
}

// 16-byte cp.async global -> shared (L2 only); valid = false zero-fills the 16 bytes
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g, bool valid)
{
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(saddr), "l"(g), "r"(n) : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                   "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                   "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
                   "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
                   "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
                   "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                   "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                   "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// MMA with both operands in shared memory, executed by a whole converged warp with
// warp-uniform operands: one lane, chosen by elect.sync, issues it (acc: accumulate or
// overwrite, warp-uniform).
__device__ __forceinline__ void umma_bf16_warp(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred e, p;\n\telect.sync _|e, 0xffffffff;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// MMA with the A operand in TMEM (K-major, two 16-bit elements per 32-bit column, the lower
// K index in the low half) and B in shared memory, executed by a whole warp with
// warp-uniform operands: one lane, chosen by elect.sync, issues the MMA.  Issued this way (operands in uniform registers) an MMA of
// M = 128, N = 32, K = 16 costs ~17 cycles; from one thread of a divergent branch ~60.
template <int ACC>
__device__ __forceinline__ void umma_bf16_ts_warp(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc)
{
    asm volatile("{\n\t.reg .pred e, p;\n\telect.sync _|e, 0xffffffff;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n"
                 :: "r"(d_tmem), "r"(a_tmem), "l"(b), "r"(idesc), "n"(ACC));
}

// tcgen05.commit from a whole warp (one elected lane)
__device__ __forceinline__ void umma_commit_warp(uint32_t mbar)
{
    asm volatile("{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
                 "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}\n"
                 :: "r"(mbar) : "memory");
}

// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes from registers; then
// tcgen05.wait::st before the data is used
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
                 "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                    "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
                    "r"(v[15])
                 : "memory");
}

// Tensor TMA through a tensor map (param, const or global space): a 3-D box into this
// CTA's shared memory (completion counted in bytes on the mbarrier), and from shared memory
// back to global memory (a bulk async-group of the issuing thread).  The innermost
// coordinate times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(uint64_t tmap, uint32_t dst, int x, int y, int z, uint32_t mbar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(mbar) : "memory");
}

__device__ __forceinline__ void tma_store_3d(uint64_t tmap, uint32_t src, int x, int y, int z)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];"
                 :: "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(src) : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// this thread's bulk stores have finished reading shared memory / have completed
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// 8 consecutive FP32 columns of this warp's 32 TMEM lanes, without the wait: several
// loads are issued, then tmem_wait_ld() makes all of them usable
__device__ __forceinline__ void tmem_ld8_async(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

// Wait for this thread's TMEM loads; the registers pass through the statement so that no
// use of them is scheduled before it.
template <int R, int C>
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[R][C])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) asm volatile("" : "+r"(v[r][c]));
}

// hi/lo split of two values into packed 16-bit pairs: hi = rn(x), lo = rn(x - hi)
__device__ __forceinline__ void split2(float a, float b, int f16, uint32_t &hi, uint32_t &lo)
{
    if (f16) {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}

// K-major, 128B swizzle: byte offset of element (row m, k) in an [128][64] bf16 plane
// Same descriptor with the 64-byte swizzle (K-major rows of 32 16-bit elements).
__device__ __forceinline__ uint64_t umma_desc_sw64(uint32_t saddr, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;    // leading byte offset: unused for swizzled K-major
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;    // SWIZZLE_64B
    return d;
}

// ... with both strides given (an MN-major operand: LBO between 32-element MN atoms, SBO
// between groups of 8 K rows)
__device__ __forceinline__ uint64_t umma_desc_sw64_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;    // SWIZZLE_64B
    return d;
}

// K-major, 64B swizzle: byte offset of the 16-byte chunk (0..3) of row m in an
// [128][32] 16-bit plane (8-row atoms of 512 bytes; chunk XOR bits 1-2 of the row)
__device__ __forceinline__ uint32_t a_off64(int m, int chunk16)
{
    return (uint32_t)((m >> 3) * 512 + (m & 7) * 64 + ((chunk16 ^ ((m & 7) >> 1)) << 4));
}

__device__ __forceinline__ uint32_t a_off(int m, int chunk16)
{
    return (uint32_t)((m >> 3) * 1024 + (m & 7) * 128 + ((chunk16 ^ (m & 7)) << 4));
}

// MN-major, 128B swizzle: byte offset of the 16-byte chunk holding columns
// n0..n0+7 (n0 multiple of 8) of K row r in a [64 K][128 N] bf16 plane
__device__ __forceinline__ uint32_t b_off(int r, int n0)
{
    const int c = (n0 & 63) >> 3;
    return (uint32_t)((r >> 3) * kBSbo + (n0 >> 6) * kBLbo + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

}  // namespace qmc
