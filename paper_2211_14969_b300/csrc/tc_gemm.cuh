// Trailing update on the 5th-generation tensor cores (tcgen05):
//   C[r0:r1, c0:c0+cw] -= L21 * U12
// with L21 taken from the shared panel (column-major, ld ldp) and U12 from
// the shared chunk Us (row-major K x CH).  Per 128-row tile the operands are
// written to shared memory in the canonical K-major, no-swizzle layout (core
// matrices of 8 rows x 16 bytes), split into a high and a low part in the
// MMA input type, and three MMAs per K-step (hi*hi + hi*lo + lo*hi)
// accumulate in FP32 in tensor memory; this keeps the product close to FP32
// accuracy while the tensor core sees only TF32 / BF16 inputs.  One thread
// issues the MMAs and commits them to an mbarrier; every warp then reads its
// 32 rows of the 128 x 64 accumulator (tcgen05.ld.32x32b.x32, twice) and updates C
// in global memory.  Waits on the mbarrier are bounded: on a timeout the
// tile is skipped and *err is set, so the caller can report the leaf.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hps {
namespace tc {

constexpr int KIND_TF32 = 1, KIND_BF16 = 2;
constexpr int TM = 128, TN = 64;  // MMA tile: 128 rows of C x 64 columns

template <int KIND> struct In;
template <> struct In<KIND_TF32> { static constexpr int BYTES = 4, KSTEP = 8; };
template <> struct In<KIND_BF16> { static constexpr int BYTES = 2, KSTEP = 16; };

// bytes of the operand buffers for a K = nb panel: A hi/lo (TM x nb), B hi/lo (TN x nb)
template <int KIND>
__host__ __device__ constexpr size_t operand_bytes(int nb) {
    return (size_t)2 * (TM + TN) * nb * In<KIND>::BYTES;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) in a K-major no-swizzle tile with K = kt
template <int KIND>
__device__ __forceinline__ int kmajor_off(int row, int k, int kt) {
    constexpr int B = In<KIND>::BYTES, PER = 16 / B;  // elements of one core-matrix row
    return (row >> 3) * (kt / PER) * 128 + (k / PER) * 128 + (row & 7) * 16 + (k % PER) * B;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; base offset 0, no swizzle
    return d;
}

template <int KIND>
__device__ __forceinline__ uint32_t instr_desc() {
    // D in FP32; A, B: TF32 (2) for kind::tf32, BF16 (1) for kind::f16;
    // both K-major; N >> 3 and M >> 4
    constexpr uint32_t fmt = KIND == KIND_TF32 ? 2u : 1u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// One 16-byte core-matrix row: PER consecutive-k values split into the high
// and low parts, written with two 16-byte stores.
template <int KIND> struct SplitRow;
template <> struct SplitRow<KIND_TF32> {
    static constexpr int PER = 4;
    __device__ static void store(unsigned char *hi, unsigned char *lo, const float *x) {
        float4 h, l;
        float *ph = (float *)&h, *pl = (float *)&l;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            ph[t] = __uint_as_float(__float_as_uint(x[t]) & 0xFFFFE000u);
            pl[t] = x[t] - ph[t];
        }
        *(float4 *)hi = h;
        *(float4 *)lo = l;
    }
};
template <> struct SplitRow<KIND_BF16> {
    static constexpr int PER = 8;
    __device__ static void store(unsigned char *hi, unsigned char *lo, const float *x) {
        uint4 h, l;
        __nv_bfloat16 *ph = (__nv_bfloat16 *)&h, *pl = (__nv_bfloat16 *)&l;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            ph[t] = __float2bfloat16_rn(x[t]);
            pl[t] = __float2bfloat16_rn(x[t] - __bfloat162float(ph[t]));
        }
        *(uint4 *)hi = h;
        *(uint4 *)lo = l;
    }
};

// Per-CTA tensor-core state in shared memory.
struct TcState {
    unsigned char *a_hi, *a_lo, *b_hi, *b_lo;
    uint64_t *mbar;
    uint32_t *tmem;    // allocated TMEM base column
    uint32_t *phase;   // mbarrier phase of the next wait
    int *err;
};

__device__ __forceinline__ void tmem_alloc(const TcState &s) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(s.tmem)),
                     "n"(TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(s.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *s.phase = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_free(const TcState &s) {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(*s.tmem), "n"(TN));
}

// bounded wait for the committed MMAs; returns false on timeout
__device__ __forceinline__ bool wait_mma(const TcState &s, uint32_t phase) {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it) {
        asm volatile(
            "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(s.mbar)), "r"(phase));
    }
    return done != 0;
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void ld_row32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc, int kind) {
    if (kind == KIND_TF32)
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                     "l"(da), "l"(db), "r"(idesc), "r"(acc));
    else
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                     "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

}  // namespace tc
}  // namespace hps
