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
// slice row is K-contiguous), integer bit operations only, each slice plane
// stored in 8 x 8 core-matrix tiles; then the GEMM: one CTA of 256 threads
// per 128 x 64 output tile, K in chunks of 16, each chunk's eight A and
// eight B slices (48 KB) loaded as two TMA boxes (cp.async.bulk.tensor,
// arrival on an mbarrier) straight into the K-major no-swizzle layout of the
// MMA operands, four buffers (two chunks' MMAs queued while the next two
// load), eight accumulators of 64 columns in TMEM (all 512 columns: one CTA
// per SM), one thread issuing the MMAs, bounded mbarrier waits (a timeout
// skips the tile and sets the error flag), and the epilogue staged through
// shared memory for row-contiguous writes.  Without the driver's tensor-map
// encoder the same loads run as cp.async.
#include <cuda.h>   // CUtensorMap and cuTensorMapEncodeTiled's types (called through the runtime's entry point)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdlib>
#include <mutex>

#include "hps_internal.cuh"
#include "merge.cuh"
#include "tc_gemm.cuh"

namespace hps {
namespace {

constexpr int OZ_S = 8;       // slices per operand
constexpr int OZ_KC = 16;     // K-chunk staged in shared memory (one MMA K-step)
constexpr int OZ_NBUF = 4;    // chunk buffers in flight
constexpr int OZ_KALIGN = 64; // K padding: a multiple of OZ_KC and of the B-slicing tile

// Slice planes are stored in 8 x 8 tiles (8 rows, 8 consecutive k: 128
// contiguous bytes), a row of tiles after the other: exactly the K-major
// no-swizzle core-matrix layout of the MMA operands, so one chunk of a
// 128-row block is 16 runs of 256 contiguous bytes (one TMA box).
__host__ __device__ __forceinline__ long long oz_tile_off(int P, int k, int Kp) {
    return ((long long)(P >> 3) * (Kp / 8) + (k >> 3)) * 64 + (P & 7) * 8 + (k & 7);
}
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
// for inf, and the slicing kernels give it to any row / column holding a
// NaN or inf; the epilogue writes NaN where a row's or column's scale is
// OZ_NONFINITE).
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

// A slices: row P of A (a gathered child row, its shared-edge columns, or a
// strided row).  As[s][P][k] (rows padded to Mp, K to Kp with zeros),
// Ea[P]; a warp per row, 8 consecutive k per lane.
__global__ void __launch_bounds__(256) oz_slice_a(OzJob J, OzakiScratch Z) {
    const int s = blockIdx.y;
    const int P = (blockIdx.x * 256 + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (P >= Z.Mp) return;
    const long long stride = (long long)Z.Mp * Z.Kp;
    __nv_bfloat16 *plane = Z.As + (long long)s * OZ_S * stride;
    const double *tr = nullptr;
    const int *s3 = nullptr;   // gathered rows: the row's entries at s3[k]
    int e = 0;
    if (P < J.M) {
        if (J.gather) {
            const MergeLevelDev &L = J.L;
            const ChildRef A = child_ref(L, L.ca[s]), B = child_ref(L, L.cb[s]);
            const int chi = L.par_child[P];
            const ChildRef &X = chi == 0 ? A : B;
            s3 = chi == 0 ? L.s3a : L.s3b;
            tr = X.T + (long long)L.par_idx[P] * X.ld;
        } else {
            tr = J.a + (long long)s * J.sa + (long long)P * J.lda;
        }
        double mx = 0.0;
        bool bad = false;   // fmax drops NaN: non-finite entries are flagged on their own
        for (int k = lane; k < J.K; k += 32) {
            const double v = tr[s3 ? s3[k] : k];
            mx = fmax(mx, fabs(v));
            bad |= !isfinite(v);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        e = __any_sync(0xffffffffu, bad) ? OZ_NONFINITE : oz_exp(mx);
    }
    for (int g = lane; g < Z.Kp / 8; g += 32) {
        double x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = g * 8 + i;
            x[i] = (tr && k < J.K) ? tr[s3 ? s3[k] : k] : 0.0;
        }
        oz_store8(x, e, plane + oz_tile_off(P, g * 8, Z.Kp), stride);
    }
    if (lane == 0) Z.Ea[(long long)s * Z.Mp + P] = e;
}

// B column exponents over the K rows: 32 columns per block, each column's
// rows split over the 8 warps (coalesced along the columns), then combined.
__global__ void __launch_bounds__(256) oz_colexp_b(OzJob J, OzakiScratch Z) {
    __shared__ double smx[8][32];
    __shared__ int sbad[8][32];
    const int s = blockIdx.y, cc = threadIdx.x & 31, rs = threadIdx.x >> 5, c = blockIdx.x * 32 + cc;
    double mx = 0.0;
    bool bad = false;   // fmax drops NaN: non-finite entries are flagged on their own
    if (c < J.N) {
        const double *b = J.b + (long long)s * J.sb + c;
        for (int k = rs; k < J.K; k += 8) {
            const double v = b[(long long)k * J.ldb];
            mx = fmax(mx, fabs(v));
            bad |= !isfinite(v);
        }
    }
    smx[rs][cc] = mx;
    sbad[rs][cc] = bad;
    __syncthreads();
    if (rs == 0 && c < Z.Np) {
        for (int r = 1; r < 8; ++r) {
            mx = fmax(mx, smx[r][cc]);
            bad |= sbad[r][cc] != 0;
        }
        Z.Fb[(long long)s * Z.Np + c] = bad ? OZ_NONFINITE : oz_exp(mx);
    }
}

// B slices Bs[t][c][k] (K-contiguous) from a 64 (k) x 32 (c) shared tile;
// a thread per (column, 8 consecutive k).
__global__ void __launch_bounds__(256) oz_slice_b(OzJob J, OzakiScratch Z) {
    __shared__ double tile[64][33];
    const int s = blockIdx.z, c0 = blockIdx.x * 32, k0 = blockIdx.y * 64;
    const double *b = J.b + (long long)s * J.sb;
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
        const int kk = e >> 5, cc = e & 31, k = k0 + kk, c = c0 + cc;
        tile[kk][cc] = (k < J.K && c < J.N) ? b[(long long)k * J.ldb + c] : 0.0;
    }
    __syncthreads();
    const int cc = threadIdx.x >> 3, g = threadIdx.x & 7, c = c0 + cc;
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = tile[g * 8 + i][cc];
    const long long stride = (long long)Z.Np * Z.Kp;
    oz_store8(x, Z.Fb[(long long)s * Z.Np + c], Z.Bs + (long long)s * OZ_S * stride + oz_tile_off(c, k0 + g * 8, Z.Kp),
              stride);
}

__device__ __forceinline__ uint32_t oz_smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void oz_cp16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(oz_smem_addr(dst)), "l"(src) : "memory");
}

// one lane of a converged warp (the MMA and TMA issues run from warp 0 as a
// whole, so their descriptors stay warp-uniform)
__device__ __forceinline__ bool oz_elect() {
    uint32_t p = 0;
    asm volatile("{\n.reg .pred q;\nelect.sync _|q, 0xffffffff;\nselp.u32 %0, 1, 0, q;\n}\n" : "=r"(p));
    return p != 0;
}

__device__ __forceinline__ void oz_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(oz_smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// one TMA box of a 3-D tensor map into shared memory, arrival on mbar
__device__ __forceinline__ void oz_tma3(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(oz_smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(oz_smem_addr(mbar))
        : "memory");
}

// bounded wait on an mbarrier phase
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

// X 2^e rounded to nearest (ties to even), built from the bits of the
// int64 X (|X| < 2^63) with integer operations; ldexp outside the normal
// range.
__device__ __forceinline__ double oz_scaled_i64(long long X, int e) {
    if (X == 0) return 0.0;
    const unsigned long long sg = X < 0 ? 1ull << 63 : 0ull;
    unsigned long long u = X < 0 ? (unsigned long long)(-X) : (unsigned long long)X;
    const int lz = __clzll((long long)u);
    u <<= lz;                                   // leading one at bit 63
    unsigned long long m = u >> 11;             // 53 significant bits
    const unsigned long long rem = u & 0x7FFull;
    if (rem > 0x400ull || (rem == 0x400ull && (m & 1ull))) ++m;
    int ex = 63 - lz + e;                       // X 2^e = (m / 2^52) 2^ex
    if (m >> 53) { m >>= 1; ++ex; }
    const int be = ex + 1023;
    if (be <= 0 || be >= 2047) return ldexp((double)X, e);
    return __longlong_as_double((long long)(sg | ((unsigned long long)be << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// t 2^e for a float t that is zero or normal, by moving its exponent and
// mantissa into a double (exact); ldexp outside the normal range.
__device__ __forceinline__ double oz_scaled_f32(float t, int e) {
    const unsigned b = __float_as_uint(t);
    const int fe = (int)((b >> 23) & 0xFF);
    if (fe == 0) return 0.0;
    const int be = fe - 127 + e + 1023;
    if (fe == 0xFF || be <= 0 || be >= 2047) return ldexp((double)t, e);
    return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) | ((unsigned long long)be << 52) |
                                            ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

// Exactness periods of the FP32 accumulators, in K-chunks of OZ_KC = 16:
// D_d over K columns is a sum of at most (d + 1) K products of magnitude
// <= 127^2, exact while (d + 1) K 127^2 < 2^24, i.e. K <= 1024, 512, 256,
// 256, 128, 128 for d = 0..5.  D_6 and D_7 (weights 2^-56, 2^-63) stay in
// tensor memory over the whole K: their FP32 rounding is below the FP64
// product's own error bound.
__device__ __forceinline__ int oz_period(int d) {
    return d == 0 ? 64 : d == 1 ? 32 : d <= 3 ? 16 : d <= 5 ? 8 : 1 << 30;
}
__device__ __forceinline__ bool oz_folds(int d, int c, int nc) { return (c + 1) % oz_period(d) == 0 || c == nc - 1; }

// (A B)[P][c] = 2^(Ea_P + Fb_c) (2^-49 X + 2^-56 (D_6 + 2^-7 D_7)),
// X = sum_{d <= 5} D_d 2^(7 (5 - d)) in exact int64 fixed point; the
// epilogue writes the merge's Th = G + A B or updates C -= A B in place.
// Chunk c: the 36 products of its eight A and eight B slices (36 MMAs of
// K = 16), from buffer c % OZ_NBUF; chunk c + 2's loads are issued once
// chunk c - 2's MMAs are done, so two chunks' MMAs stay queued, except
// after a chunk whose accumulators are folded.
__global__ void __launch_bounds__(OZ_NT, 1) oz_gemm(OzJob J, OzakiScratch Z, const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB) {
    extern __shared__ __align__(1024) unsigned char smem[];
    using namespace tc;
    constexpr int BSL = OZ_TN * OZ_KC * 2;           // one B slice tile, bytes
    constexpr int ASL = OZ_TM * OZ_KC * 2;           // one A slice tile
    constexpr int BUF = OZ_S * (ASL + BSL);          // one chunk: 8 A + 8 B slices
    uint64_t *mbar = (uint64_t *)(smem + OZ_NBUF * BUF);   // [OZ_NBUF] MMA completion, one per buffer
    uint64_t *full = mbar + OZ_NBUF;                       // [OZ_NBUF] TMA arrival, one per buffer
    uint32_t *tmem_p = (uint32_t *)(full + OZ_NBUF);
    const int s = blockIdx.z, tm = blockIdx.y * OZ_TM, tn = blockIdx.x * OZ_TN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;     // TMEM lanes 32 quad.., columns 32 half..
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(oz_smem_addr(tmem_p)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int b = 0; b < OZ_NBUF; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(oz_smem_addr(mbar + b)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(oz_smem_addr(full + b)));
        }
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
    const int nc = Z.Kp / OZ_KC;
    // chunk c's slices into buffer c % OZ_NBUF (A slices first, then B): one
    // TMA box each, issued by thread 0 (arrival on full[]), or without a
    // tensor map cp.async of the same 256-byte runs by every thread
    int issued = 0;   // chunks whose loads were issued
    auto load_chunk = [&](int c) {
        unsigned char *buf = smem + (c % OZ_NBUF) * BUF;
        const int kc = c * OZ_KC;
        issued = c + 1;
        if (Z.tma) {
            if (warp == 0 && oz_elect()) {
                oz_expect_tx(full + c % OZ_NBUF, BUF);
                oz_tma3(buf, &tmA, kc * 8, tm / 8, s * OZ_S, full + c % OZ_NBUF);
                oz_tma3(buf + OZ_S * ASL, &tmB, kc * 8, tn / 8, s * OZ_S, full + c % OZ_NBUF);
            }
            return;
        }
        constexpr int RUN = OZ_KC;                   // 16-byte pieces per 256-byte run (one 8-row block)
        for (int e = tid; e < OZ_S * (OZ_TM / 8) * RUN; e += OZ_NT) {
            const int sl = e / ((OZ_TM / 8) * RUN), r = e % ((OZ_TM / 8) * RUN), ph = r / RUN, j = r % RUN;
            oz_cp16(buf + sl * ASL + ph * RUN * 16 + j * 16, Ag + sl * sa + oz_tile_off(tm + ph * 8, kc, Z.Kp) + j * 8);
        }
        for (int e = tid; e < OZ_S * (OZ_TN / 8) * RUN; e += OZ_NT) {
            const int t = e / ((OZ_TN / 8) * RUN), r = e % ((OZ_TN / 8) * RUN), ph = r / RUN, j = r % RUN;
            oz_cp16(buf + OZ_S * ASL + t * BSL + ph * RUN * 16 + j * 16,
                    Bg + t * sb + oz_tile_off(tn + ph * 8, kc, Z.Kp) + j * 8);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    // chunk c's MMAs complete (the k-th completion of barrier b is chunk c = b + OZ_NBUF k)
    int waited = -1;
    auto wait_chunk = [&](int c) -> bool {
        if (c <= waited) return true;
        waited = c;
        return oz_wait(mbar + c % OZ_NBUF, (uint32_t)((c / OZ_NBUF) & 1));
    };
    long long X[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) X[c] = 0;
    const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + half * 32;
    auto fold = [&](int c) {
#pragma unroll 1
        for (int d = 0; d < 6; ++d) {
            if (!oz_folds(d, c, nc)) continue;
            float v[32];
            ld_row32(trow + d * OZ_TN, v);
            const long long w = 1LL << (7 * (5 - d));
#pragma unroll
            for (int j = 0; j < 32; ++j) X[j] += (long long)__float2int_rn(v[j]) * w;
        }
    };
    bool ok = true, mine = true;
    int consumed = 0;   // chunks whose arrival thread 0 waited for (TMA)
    for (int c = 0; c < OZ_NBUF - 2 && c < nc; ++c) load_chunk(c);
    for (int c = 0; c < nc; ++c) {
        if (Z.tma) {   // thread 0 issues the MMAs: it alone waits for the chunk's arrival
            if (warp == 0) mine = mine && oz_wait(full + c % OZ_NBUF, (uint32_t)((c / OZ_NBUF) & 1));
            if (warp == 0) consumed = c + 1;
        } else {       // chunk c's group complete; chunk c + 1's may be in flight
            if (c + 1 < nc) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        bool folded = false;
        for (int d = 0; d < 6 && c >= 1; ++d) folded |= oz_folds(d, c - 1, nc);
        // with TMA only thread 0 touches a chunk before its MMAs, so the CTA
        // meets only where it folds; with cp.async every thread's copies of
        // the chunk must be visible first
        if (!Z.tma || folded) {
            if (!Z.tma) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            ok = __syncthreads_and(mine) != 0;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (!ok) break;
        }
        if (folded) {   // chunk c - 1's accumulators are read before chunk c resets them
            ok = __syncthreads_and(wait_chunk(c - 1)) != 0;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (!ok) break;
            fold(c - 1);
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        }
        if (warp == 0 && __all_sync(0xffffffffu, mine)) {
            // descriptors are linear in the address (its >> 4 in the low bits):
            // every MMA's is a base plus a compile-time offset; warp 0 holds
            // them uniformly and one elected lane issues
            const uint32_t a0 = oz_smem_addr(smem + (c % OZ_NBUF) * BUF), b0 = a0 + OZ_S * ASL;
            const uint64_t da0 = smem_desc(a0, lbo, sbo), db0 = smem_desc(b0, lbo, sbo);
            uint32_t keep = 0;   // bit d: chunk c continues D_d's period
#pragma unroll
            for (int d = 0; d < OZ_S; ++d) keep |= (c % oz_period(d) != 0 ? 1u : 0u) << d;
            if (oz_elect()) {
#pragma unroll
            for (int sl = 0; sl < OZ_S; ++sl) {
#pragma unroll
                for (int t = 0; t < OZ_S - sl; ++t) {
#pragma unroll
                    for (int ks = 0; ks < OZ_KC / 16; ++ks) {
                        const uint64_t da = da0 + (uint64_t)((sl * ASL + ks * 256) >> 4);
                        const uint64_t db = db0 + (uint64_t)((t * BSL + ks * 256) >> 4);
                        const uint32_t acc = (sl == 0 && ks == 0) ? (keep >> t) & 1u : 1u;
                        mma(tmem + (sl + t) * OZ_TN, da, db, idesc, acc, KIND_BF16);
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                oz_smem_addr(mbar + c % OZ_NBUF)));
            }
            __syncwarp();
        }
        // chunk c - 2 (long done: the MMAs of chunks c - 1 and c stay queued)
        // frees the buffer chunk c + OZ_NBUF - 2 loads into
        if (c >= 2 && (!Z.tma || warp == 0)) mine = mine && wait_chunk(c - 2);
        if (c + OZ_NBUF - 2 < nc && mine) load_chunk(c + OZ_NBUF - 2);
    }
    if (ok) {   // agree that every wait succeeded before waiting for the last chunk's MMAs
        ok = __syncthreads_and(mine) != 0;
        if (ok) ok = __syncthreads_and(wait_chunk(nc - 1)) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (ok) fold(nc - 1);
    }
    if (!ok && tid == 0) atomicExch(Z.err, 1);
    if (!ok && Z.tma && warp == 0)   // boxes still in flight land before the CTA ends (bounded)
        for (int c = consumed; c < issued; ++c) oz_wait(full + c % OZ_NBUF, (uint32_t)((c / OZ_NBUF) & 1));
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    // this thread's 32 products (X and the FP32 tail D_6 + 2^-7 D_7),
    // staged for row-wise writes (the slice buffers are free)
    constexpr int SLD = OZ_TN + 1;
    long long *stX = (long long *)smem;                              // [OZ_TM][SLD]
    float *stT = (float *)(smem + (size_t)OZ_TM * SLD * sizeof(long long));   // [OZ_TM][SLD]
    if (ok) {
        float v6[32], v7[32];
        ld_row32(trow + 6 * OZ_TN, v6);
        ld_row32(trow + 7 * OZ_TN, v7);
        const int r = quad * 32 + lane;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            stX[r * SLD + half * 32 + c] = X[c];
            stT[r * SLD + half * 32 + c] = v6[c] + v7[c] * 0x1p-7f;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
    if (!ok) return;
    // epilogue: warp w takes rows w, w + 8, ..; lanes the columns lane, lane + 32
    const MergeLevelDev &L = J.L;
    ChildRef A{}, B{};
    if (J.form) {
        A = child_ref(L, L.ca[s]);
        B = child_ref(L, L.cb[s]);
    }
    constexpr int RW = OZ_TM / (OZ_NT / 32);   // rows per warp (16)
    int pc[2], pi[2], fb[2];
    bool cv[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int col = tn + u * 32 + lane;
        cv[u] = col < J.N;
        pc[u] = (J.form && col < L.np) ? L.par_child[col] : -1;   // -1: a load column of h
        pi[u] = (J.form && col < L.np) ? L.par_idx[col] : col - L.np;
        fb[u] = cv[u] ? Z.Fb[(long long)s * Z.Np + col] : 0;
    }
    int rchi = 0, ridx = 0, rea = 0;
    if (lane < RW) {
        const int P = tm + warp + (OZ_NT / 32) * lane;
        if (P < J.M) {
            if (J.form) {
                rchi = L.par_child[P];
                ridx = L.par_idx[P];
            }
            rea = Z.Ea[(long long)s * Z.Mp + P];
        }
    }
    // the gathered part G (the merge) or C (an update) of every row first, then the stores
    double gv[RW][2];
#pragma unroll
    for (int i = 0; i < RW; ++i) {
        const int P = tm + warp + (OZ_NT / 32) * i;
        const int chi = __shfl_sync(0xffffffffu, rchi, i), idx = __shfl_sync(0xffffffffu, ridx, i);
        const ChildRef &Xc = chi == 0 ? A : B;
        const double *crow = J.c + (long long)s * J.sc + (long long)P * J.ldc + tn;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            double g = 0.0;
            if (P < J.M && cv[u]) {
                if (!J.form) g = crow[u * 32 + lane];
                else if (pc[u] < 0) g = Xc.h[(long long)idx * Xc.ldh + pi[u]];
                else if (pc[u] == chi) g = Xc.T[(long long)idx * Xc.ld + pi[u]];
            }
            gv[i][u] = g;
        }
    }
    const double sign = J.form ? 1.0 : -1.0;
#pragma unroll
    for (int i = 0; i < RW; ++i) {
        const int r = warp + (OZ_NT / 32) * i, P = tm + r;
        const int ea = __shfl_sync(0xffffffffu, rea, i);
        if (P >= J.M) break;
        double *out = J.c + (long long)s * J.sc + (long long)P * J.ldc + tn;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (!cv[u]) continue;
            const int c = u * 32 + lane, sc = ea + fb[u];
            double v;
            if (ea >= OZ_NONFINITE || fb[u] >= OZ_NONFINITE) v = __longlong_as_double(0x7FF8000000000000LL);
            else v = fma(sign, oz_scaled_i64(stX[r * SLD + c], sc - 49) + oz_scaled_f32(stT[r * SLD + c], sc - 56), gv[i][u]);
            out[c] = v;
        }
    }
}

}  // namespace

size_t ozaki_scratch_bytes(int nm, int M, int K, int N) {
    const long long Kp = (K + OZ_KALIGN - 1) / OZ_KALIGN * OZ_KALIGN;
    const long long Mp = (M + OZ_TM - 1) / OZ_TM * OZ_TM, Np = (N + OZ_TN - 1) / OZ_TN * OZ_TN;
    return (size_t)nm * (OZ_S * (Mp + Np) * Kp * 2 + (Mp + Np) * 4) + 256;
}

// K <= 8192 keeps the int64 fixed-point sum of the D_d below 2^63
bool ozaki_applies(int np, int n3) { return n3 >= 16 && n3 <= 8192 && np >= 64; }

OzakiScratch ozaki_layout(void *base, int nm, int M, int K, int N, int *err) {
    OzakiScratch Z{};
    Z.Kp = (K + OZ_KALIGN - 1) / OZ_KALIGN * OZ_KALIGN;
    Z.Mp = (M + OZ_TM - 1) / OZ_TM * OZ_TM;
    Z.Np = (N + OZ_TN - 1) / OZ_TN * OZ_TN;
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

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, through the runtime (null if unavailable,
// or when the environment sets HPS_OZAKI_TMA=0: the GEMM then loads with
// cp.async); looked up once per process
static EncodeTiled encode_tiled() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *env = getenv("HPS_OZAKI_TMA");
        if (env && env[0] == '0') return;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
    });
    return fn;
}

cudaError_t launch_ozaki(const OzJob &J, const OzakiScratch &Z0, cudaStream_t st) {
    if (J.M <= 0 || J.N <= 0 || J.K <= 0) return cudaSuccess;
    // the layout for this job's sizes, in the same scratch (sized for the largest job)
    OzakiScratch Z = ozaki_layout(Z0.As, J.nm, J.M, J.K, J.N, Z0.err);
    oz_slice_a<<<dim3((Z.Mp * 32 + 255) / 256, J.nm), 256, 0, st>>>(J, Z);
    oz_colexp_b<<<dim3(Z.Np / 32, J.nm), 256, 0, st>>>(J, Z);
    oz_slice_b<<<dim3(Z.Np / 32, Z.Kp / 64, J.nm), 256, 0, st>>>(J, Z);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = OZ_NBUF * (size_t)OZ_S * (OZ_TM + OZ_TN) * OZ_KC * 2 + 128;
    e = cudaFuncSetAttribute(oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // tensor maps of the two slice arrays: (k within a row of tiles, row block, slice plane)
    CUtensorMap tmA{}, tmB{};
    Z.tma = 0;
    if (EncodeTiled fn = encode_tiled()) {
        const cuuint32_t boxA[3] = {OZ_KC * 8, OZ_TM / 8, OZ_S}, boxB[3] = {OZ_KC * 8, OZ_TN / 8, OZ_S}, es[3] = {1, 1, 1};
        const cuuint64_t dA[3] = {(cuuint64_t)Z.Kp * 8, (cuuint64_t)Z.Mp / 8, (cuuint64_t)J.nm * OZ_S};
        const cuuint64_t dB[3] = {(cuuint64_t)Z.Kp * 8, (cuuint64_t)Z.Np / 8, (cuuint64_t)J.nm * OZ_S};
        const cuuint64_t sA[2] = {(cuuint64_t)Z.Kp * 16, (cuuint64_t)Z.Mp * Z.Kp * 2};
        const cuuint64_t sB[2] = {(cuuint64_t)Z.Kp * 16, (cuuint64_t)Z.Np * Z.Kp * 2};
        const bool okA = fn(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Z.As, dA, sA, boxA, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        const bool okB = okA && fn(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Z.Bs, dB, sB, boxB, es,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        Z.tma = okA && okB;
    }
    oz_gemm<<<dim3(Z.Np / OZ_TN, Z.Mp / OZ_TM, J.nm), OZ_NT, smem, st>>>(J, Z, tmA, tmB);
    return cudaGetLastError();
}

cudaError_t launch_parent_ozaki(const MergeLevelDev &L, const OzakiScratch &Z, cudaStream_t st) {
    OzJob J{};
    J.nm = L.nm;
    J.M = L.np;
    J.K = L.n3;
    J.N = L.np + L.m;
    J.gather = 1;
    J.b = L.aug + L.c3;
    J.sb = (long long)L.n3 * L.lda;
    J.ldb = L.lda;
    J.form = 1;
    J.c = L.Th;
    J.ldc = L.np + L.m;
    J.sc = (long long)L.np * J.ldc;
    J.L = L;
    return launch_ozaki(J, Z, st);
}

}  // namespace hps
