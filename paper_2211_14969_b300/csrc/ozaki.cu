// The parents' [T | h] of the upper merge levels as an FP64-accurate product
// on the BF16 tensor cores (tcgen05), by splitting the FP64 operands into
// exact integer slices (the error-free splitting of Ozaki, Ogita, Oishi and
// Rump, 2012, with per-row and per-column power-of-two scales).
//
// The merge forms per merge (Section 2 of arXiv 2211.14969, from its HPS
// references) T = G + A B with A = [Ta13; Tb23] (np x n3, gathered from the
// children's maps), B = [S3 | w3] (n3 x (np + m), the solved augmented
// system) and G the gathered diag(Ta11, Tb22) | [ha1; hb2].  Here:
//   row i of A:    a_ik = 2^Ei sum_{s<8} alpha_ik^(s) 2^-7(s+1),  |alpha| <= 127
//   column j of B: b_kj = 2^Fj sum_{t<8} beta_kj^(t) 2^-7(t+1),
// (each slice an integer, exact in BF16; what is cut off is below 2^-56 of
// the row's / column's largest entry), and
//   (A B)_ij = 2^(Ei+Fj) sum_{d<8} 2^-7(d+2) D_d,  D_d = sum_{s+t=d} sum_k alpha^(s) beta^(t)
// (products with s + t >= 8 are below 2^-63 of |a||b| and dropped).  D_d
// accumulates in FP32 in tensor memory; for d <= 5 it is exact over up to
// 1024 / (d + 1) columns of K (sums of integers below 2^24) and is folded at
// that period into an exact int64 fixed-point sum; D_6 and D_7 stay in FP32
// over the whole K (their rounding is below the FP64 product's own error).
//
// Kernels: the slices of A (a warp per row, the gather included) and of B
// (column exponents, then slices transposed through shared memory so every
// slice row is K-contiguous), integer bit operations only; then the GEMM:
// one CTA of 256 threads per 128 x 64 output tile, K in chunks of 64, the
// chunk's eight B slices (8 x 64 x 64) and one A slice (128 x 64) in shared
// memory in the K-major no-swizzle core-matrix layout, both double-buffered
// so the next stage's cp.async loads overlap the current stage's MMAs, eight
// accumulators of 64 columns in TMEM (all 512 columns: one CTA per SM), one
// thread issuing the MMAs, bounded mbarrier waits (a timeout skips the tile
// and sets the error flag), and the epilogue staged through shared memory
// for row-contiguous writes.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hps_internal.cuh"
#include "merge.cuh"
#include "tc_gemm.cuh"

namespace hps {
namespace {

constexpr int OZ_S = 8;       // slices per operand
constexpr int OZ_KC = 64;     // K-chunk staged in shared memory
constexpr int OZ_TM = 128, OZ_TN = 64;
constexpr int OZ_NT = 256;

struct ChildRef {
    const double *T, *h;
    int ld, ldh;
};

__device__ __forceinline__ ChildRef child_ref(const MergeLevelDev &L, int child) {
    ChildRef v;
    if (L.leaf_T) {
        v.T = L.leaf_T + (long long)child * L.nbc * L.nbc;
        v.ld = L.nbc;
        v.h = L.leaf_h ? L.leaf_h + (long long)child * L.nbc * L.m : nullptr;
        v.ldh = L.m;
    } else {
        const long long ldc = L.nbc + L.m;
        v.T = L.prev_Th + (long long)child * L.nbc * ldc;
        v.ld = (int)ldc;
        v.h = v.T + L.nbc;
        v.ldh = (int)ldc;
    }
    return v;
}

// Scale exponent e with |x| < 2^e for every |x| <= amax, from the bits of
// amax (0 for amax == 0 or subnormal: such rows are flushed; OZ_NONFINITE
// for inf / NaN, which the epilogue turns into NaN).
constexpr int OZ_NONFINITE = 4096;
__device__ __forceinline__ int oz_exp(double amax) {
    const int ex = (int)(((unsigned long long)__double_as_longlong(amax) >> 52) & 0x7FF);
    return ex == 0 ? 0 : ex == 0x7FF ? OZ_NONFINITE : ex - 1022;
}

// trunc(|x| 2^(56 - e)) < 2^56 for |x| < 2^e: x = mant 2^(ex - 1075)
__device__ __forceinline__ unsigned long long oz_fixed(unsigned long long b, int e) {
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0 || ex == 0x7FF || e >= OZ_NONFINITE) return 0;
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = ex - 1019 - e;
    if (sh >= 0) return mant << sh;
    return sh <= -64 ? 0 : mant >> (-sh);
}

// The 8 integer slices of 8 consecutive values x (all scaled by 2^-e):
// slice s = sign(x) ((trunc(|x| 2^(56-e)) >> (49 - 7 s)) & 127), exact in
// BF16; written as one 16-byte row of 8 BF16 per slice plane.
__device__ __forceinline__ void oz_store8(const double *x, int e, __nv_bfloat16 *dst, long long stride) {
    unsigned long long V[8];
    unsigned sg[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(x[i]);
        V[i] = oz_fixed(b, e);
        sg[i] = (unsigned)(b >> 63);
    }
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t h[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int a = (int)((V[2 * i + u] >> (49 - 7 * s)) & 127);
                h[u] = __float_as_uint(__int2float_rn(sg[2 * i + u] ? -a : a)) >> 16;   // |a| <= 127: exact
            }
            w[i] = h[0] | (h[1] << 16);
        }
        *(uint4 *)(dst + s * stride) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// A slices: row P of A = the gathered child row (its shared-edge columns).
// As[s][P][k] (rows padded to Mp, K to Kp with zeros), Ea[P]; a warp per
// row, 8 consecutive k per lane.
__global__ void __launch_bounds__(256) oz_slice_a(MergeLevelDev L, OzakiScratch Z) {
    const int s = blockIdx.y;
    const int P = (blockIdx.x * 256 + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (P >= Z.Mp) return;
    const long long stride = (long long)Z.Mp * Z.Kp;
    __nv_bfloat16 *row = Z.As + (long long)s * OZ_S * stride + (long long)P * Z.Kp;
    const double *tr = nullptr;
    const int *s3 = nullptr;
    int e = 0;
    if (P < L.np) {
        const ChildRef A = child_ref(L, L.ca[s]), B = child_ref(L, L.cb[s]);
        const int chi = L.par_child[P];
        const ChildRef &X = chi == 0 ? A : B;
        s3 = chi == 0 ? L.s3a : L.s3b;
        tr = X.T + (long long)L.par_idx[P] * X.ld;
        double mx = 0.0;
        for (int k = lane; k < L.n3; k += 32) mx = fmax(mx, fabs(tr[s3[k]]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        e = oz_exp(mx);
    }
    for (int g = lane; g < Z.Kp / 8; g += 32) {
        double x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = g * 8 + i;
            x[i] = (tr && k < L.n3) ? tr[s3[k]] : 0.0;
        }
        oz_store8(x, e, row + g * 8, stride);
    }
    if (lane == 0) Z.Ea[(long long)s * Z.Mp + P] = e;
}

// B column exponents: column c of B = aug[:, c3 + c] over the n3 rows.
__global__ void __launch_bounds__(256) oz_colexp_b(MergeLevelDev L, OzakiScratch Z) {
    const int s = blockIdx.y, c = blockIdx.x * 256 + threadIdx.x;
    if (c >= Z.Np) return;
    const int N = L.np + L.m;
    double mx = 0.0;
    if (c < N) {
        const double *aug = L.aug + (long long)s * L.n3 * L.lda + L.c3 + c;
        for (int k = 0; k < L.n3; ++k) mx = fmax(mx, fabs(aug[(long long)k * L.lda]));
    }
    Z.Fb[(long long)s * Z.Np + c] = oz_exp(mx);
}

// B slices Bs[t][c][k] (K-contiguous) from a 64 (k) x 32 (c) shared tile;
// a thread per (column, 8 consecutive k).
__global__ void __launch_bounds__(256) oz_slice_b(MergeLevelDev L, OzakiScratch Z) {
    __shared__ double tile[64][33];
    const int s = blockIdx.z, c0 = blockIdx.x * 32, k0 = blockIdx.y * 64;
    const int N = L.np + L.m;
    const double *aug = L.aug + (long long)s * L.n3 * L.lda + L.c3;
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
        const int kk = e >> 5, cc = e & 31, k = k0 + kk, c = c0 + cc;
        tile[kk][cc] = (k < L.n3 && c < N) ? aug[(long long)k * L.lda + c] : 0.0;
    }
    __syncthreads();
    const int cc = threadIdx.x >> 3, g = threadIdx.x & 7, c = c0 + cc;
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = tile[g * 8 + i][cc];
    const long long stride = (long long)Z.Np * Z.Kp;
    oz_store8(x, Z.Fb[(long long)s * Z.Np + c], Z.Bs + (long long)s * OZ_S * stride + (long long)c * Z.Kp + k0 + g * 8,
              stride);
}

__device__ __forceinline__ uint32_t oz_smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void oz_cp16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(oz_smem_addr(dst)), "l"(src) : "memory");
}

// bounded wait on the MMA-completion mbarrier
__device__ __forceinline__ bool oz_wait(uint64_t *mbar, uint32_t phase) {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it) {
        asm volatile(
            "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(done)
            : "r"(oz_smem_addr(mbar)), "r"(phase));
    }
    return done != 0;
}

// Exactness periods of the FP32 accumulators, in K-chunks of OZ_KC = 64:
// D_d over K columns is a sum of at most (d + 1) K products of magnitude
// <= 127^2, exact while (d + 1) K 127^2 < 2^24, i.e. K <= 1024, 512, 256,
// 256, 128, 128 for d = 0..5.  D_6 and D_7 (weights 2^-56, 2^-63) stay in
// tensor memory over the whole K: their FP32 rounding is below the FP64
// product's own error bound.
__device__ __forceinline__ int oz_period(int d) {
    return d == 0 ? 16 : d == 1 ? 8 : d <= 3 ? 4 : d <= 5 ? 2 : 1 << 30;
}

// Th[P][c] = G[P][c] + 2^(Ea_P + Fb_c) (2^-49 X + 2^-56 (D_6 + 2^-7 D_7)),
// X = sum_{d <= 5} D_d 2^(7 (5 - d)) in exact int64 fixed point.
// Stages j = 8 ci + sl: A slice sl of K-chunk ci against the chunk's B
// slices t <= 7 - sl; A and B double-buffered, the next stage's loads in
// flight during the current stage's MMAs.
__global__ void __launch_bounds__(OZ_NT, 1) oz_gemm(MergeLevelDev L, OzakiScratch Z) {
    extern __shared__ __align__(1024) unsigned char smem[];
    using namespace tc;
    constexpr int BSL = OZ_TN * OZ_KC * 2;           // one B slice tile, bytes
    constexpr int BCH = OZ_S * BSL;                  // one chunk's B slices
    constexpr int ASL = OZ_TM * OZ_KC * 2;           // one A slice tile
    unsigned char *bs = smem;                        // [2][OZ_S] B slice tiles
    unsigned char *as = smem + 2 * BCH;              // [2] A slice tiles
    uint64_t *mbar = (uint64_t *)(as + 2 * ASL);     // [2] MMA completion, one per A buffer
    uint32_t *tmem_p = (uint32_t *)(mbar + 2);
    const int s = blockIdx.z, tm = blockIdx.y * OZ_TM, tn = blockIdx.x * OZ_TN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;     // TMEM lanes 32 quad.., columns 32 half..
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(oz_smem_addr(tmem_p)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(oz_smem_addr(mbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(oz_smem_addr(mbar + 1)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_p;
    const uint32_t idesc = instr_desc<KIND_BF16>();    // M = 128, N = 64, BF16 in, FP32 accumulate
    const uint32_t lbo = 128, sbo = (OZ_KC / 8) * 128;
    const long long sa = (long long)Z.Mp * Z.Kp, sb = (long long)Z.Np * Z.Kp;
    const __nv_bfloat16 *Ag = Z.As + (long long)s * OZ_S * sa;
    const __nv_bfloat16 *Bg = Z.Bs + (long long)s * OZ_S * sb;
    const int nc = Z.Kp / OZ_KC, NS = nc * OZ_S;
    // cp.async of stage j's A slice (and, at sl = 0, its chunk's B slices)
    auto load_stage = [&](int j) {
        const int ci = j / OZ_S, sl = j % OZ_S, kc = ci * OZ_KC;
        if (sl == 0) {
            unsigned char *bb = bs + (ci & 1) * BCH;
            for (int e = tid; e < OZ_S * OZ_TN * (OZ_KC / 8); e += OZ_NT) {
                const int t = e / (OZ_TN * (OZ_KC / 8)), r = e % (OZ_TN * (OZ_KC / 8));
                const int n = r / (OZ_KC / 8), g = r % (OZ_KC / 8);
                oz_cp16(bb + t * BSL + kmajor_off<KIND_BF16>(n, g * 8, OZ_KC),
                        Bg + t * sb + (long long)(tn + n) * Z.Kp + kc + g * 8);
            }
        }
        unsigned char *ab = as + (j & 1) * ASL;
        for (int e = tid; e < OZ_TM * (OZ_KC / 8); e += OZ_NT) {
            const int m = e / (OZ_KC / 8), g = e % (OZ_KC / 8);
            oz_cp16(ab + kmajor_off<KIND_BF16>(m, g * 8, OZ_KC), Ag + sl * sa + (long long)(tm + m) * Z.Kp + kc + g * 8);
        }
    };
    // stage j's MMAs complete (the k-th completion of barrier j & 1 is stage j = (j & 1) + 2k)
    int waited = -1;
    auto wait_stage = [&](int j) -> bool {
        if (j <= waited) return true;
        waited = j;
        return oz_wait(mbar + (j & 1), (uint32_t)((j >> 1) & 1));
    };
    long long X[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) X[c] = 0;
    const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + half * 32;
    bool ok = true;
    load_stage(0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int j = 0; j < NS; ++j) {
        const int ci = j / OZ_S, sl = j % OZ_S;
        bool mine = true;
        if (j + 1 < NS) {
            // stage j - 1 used the buffers stage j + 1 loads into
            if (j >= 1) mine = wait_stage(j - 1);
            if (mine) load_stage(j + 1);
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 1;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        ok = __syncthreads_and(mine) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!ok) break;
        if (tid == 0) {
            const uint32_t a0 = oz_smem_addr(as + (j & 1) * ASL), b0 = oz_smem_addr(bs + (ci & 1) * BCH);
            for (int t = 0; t < OZ_S - sl; ++t) {
                const int d = sl + t;
                const bool reset = sl == 0 && ci % oz_period(d) == 0;
#pragma unroll
                for (int ks = 0; ks < OZ_KC / 16; ++ks) {
                    const uint32_t step = ks * 2 * 128;
                    const uint64_t da = smem_desc(a0 + step, lbo, sbo);
                    const uint64_t db = smem_desc(b0 + t * BSL + step, lbo, sbo);
                    mma(tmem + d * OZ_TN, da, db, idesc, (reset && ks == 0) ? 0u : 1u, KIND_BF16);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                oz_smem_addr(mbar + (j & 1))));
        }
        if (sl != OZ_S - 1) continue;
        // end of chunk ci: fold the accumulators whose period ends here
        bool fold = ci == nc - 1;
        for (int d = 0; d < 6; ++d) fold |= (ci + 1) % oz_period(d) == 0;
        if (!fold) continue;
        ok = __syncthreads_and(wait_stage(j)) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!ok) break;
#pragma unroll 1
        for (int d = 0; d < 6; ++d) {
            if ((ci + 1) % oz_period(d) != 0 && ci != nc - 1) continue;
            float v[32];
            ld_row32(trow + d * OZ_TN, v);
            const int sh = 7 * (5 - d);
#pragma unroll
            for (int c = 0; c < 32; ++c) X[c] += (long long)__float2int_rn(v[c]) * (1LL << sh);
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    }
    if (!ok && tid == 0) atomicExch(Z.err, 1);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    if (ok) {
        // this thread's 32 products, staged for row-wise writes (the B buffers are free)
        double *stage = (double *)smem;   // [OZ_TM][OZ_TN + 1]
        float v6[32], v7[32];
        ld_row32(trow + 6 * OZ_TN, v6);
        ld_row32(trow + 7 * OZ_TN, v7);
        const int r = quad * 32 + lane;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const double tail = (double)v6[c] + (double)v7[c] * 0x1p-7;
            stage[r * (OZ_TN + 1) + half * 32 + c] = (double)X[c] * 0x1p-49 + tail * 0x1p-56;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
    if (!ok) return;
    // epilogue: a warp per row, lanes along its 64 columns
    const double *stage = (const double *)smem;
    const ChildRef A = child_ref(L, L.ca[s]), B = child_ref(L, L.cb[s]);
    const int ldt = L.np + L.m;
    for (int r = warp; r < OZ_TM; r += OZ_NT / 32) {
        const int P = tm + r;
        if (P >= L.np) break;
        const int chi = L.par_child[P], idx = L.par_idx[P];
        const ChildRef &Xc = chi == 0 ? A : B;
        const int ea = Z.Ea[(long long)s * Z.Mp + P];
        double *Th = L.Th + (long long)s * L.np * ldt + (long long)P * ldt;
#pragma unroll
        for (int u = 0; u < OZ_TN / 32; ++u) {
            const int c = u * 32 + lane, col = tn + c;
            if (col >= ldt) continue;
            double g;
            if (col < L.np) g = (L.par_child[col] == chi) ? Xc.T[(long long)idx * Xc.ld + L.par_idx[col]] : 0.0;
            else g = Xc.h[(long long)idx * Xc.ldh + (col - L.np)];
            const int sc = ea + Z.Fb[(long long)s * Z.Np + col];
            Th[col] = sc >= OZ_NONFINITE ? __longlong_as_double(0x7FF8000000000000LL)
                                         : g + ldexp(stage[r * (OZ_TN + 1) + c], sc);
        }
    }
}

}  // namespace

size_t ozaki_scratch_bytes(int nm, int np, int n3, int m) {
    const long long Kp = (n3 + OZ_KC - 1) / OZ_KC * OZ_KC;
    const long long Mp = (np + OZ_TM - 1) / OZ_TM * OZ_TM, Np = (np + m + OZ_TN - 1) / OZ_TN * OZ_TN;
    return (size_t)nm * (OZ_S * (Mp + Np) * Kp * 2 + (Mp + Np) * 4) + 256;
}

// n3 <= 8192 keeps the int64 fixed-point sum of the D_d below 2^63
bool ozaki_applies(int np, int n3) { return n3 >= 64 && n3 <= 8192 && np >= 2 * OZ_TM; }

OzakiScratch ozaki_layout(void *base, int nm, int np, int n3, int m, int *err) {
    OzakiScratch Z{};
    Z.Kp = (n3 + OZ_KC - 1) / OZ_KC * OZ_KC;
    Z.Mp = (np + OZ_TM - 1) / OZ_TM * OZ_TM;
    Z.Np = (np + m + OZ_TN - 1) / OZ_TN * OZ_TN;
    unsigned char *b = (unsigned char *)base;
    Z.As = (__nv_bfloat16 *)b;
    b += (size_t)nm * OZ_S * Z.Mp * Z.Kp * 2;
    Z.Bs = (__nv_bfloat16 *)b;
    b += (size_t)nm * OZ_S * Z.Np * Z.Kp * 2;
    Z.Ea = (int *)b;
    b += (size_t)nm * Z.Mp * 4;
    Z.Fb = (int *)b;
    Z.err = err;
    return Z;
}

cudaError_t launch_parent_ozaki(const MergeLevelDev &L, const OzakiScratch &Z, cudaStream_t st) {
    oz_slice_a<<<dim3((Z.Mp * 32 + 255) / 256, L.nm), 256, 0, st>>>(L, Z);
    oz_colexp_b<<<dim3((Z.Np + 255) / 256, L.nm), 256, 0, st>>>(L, Z);
    oz_slice_b<<<dim3(Z.Np / 32, Z.Kp / 64, L.nm), 256, 0, st>>>(L, Z);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = 2 * (size_t)OZ_S * OZ_TN * OZ_KC * 2 + 2 * (size_t)OZ_TM * OZ_KC * 2 + 64;
    e = cudaFuncSetAttribute(oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    oz_gemm<<<dim3(Z.Np / OZ_TN, Z.Mp / OZ_TM, L.nm), OZ_NT, smem, st>>>(L, Z);
    return cudaGetLastError();
}

}  // namespace hps
