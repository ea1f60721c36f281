// Blocked dense LU with partial pivoting on an augmented row-major matrix
// [A | 0 | RHS], run by one CTA of NT = 128 threads.
//
// Per panel of NB columns:
//   * the panel (rows k0..n-1) is staged in shared memory (column-major) and
//     factored there: warp-shuffle argmax per column, row swap, scaling and
//     rank-1 update of the remaining panel columns;
//   * the panel's row interchanges are turned into one permutation of the
//     touched rows, applied to the columns right of the panel by gathering
//     the source rows (no serial swap chains through global memory);
//   * the unit-lower solve U12 = L11^{-1} A12 runs one column per thread
//     with the column held in registers;
//   * the trailing update A22 -= L21 U12 is register-tiled (2HV x 2HV per
//     thread, 16-byte vector loads from shared and global memory).
// Then U X = Y is solved in place for the right-hand columns by block rows
// from the bottom with the same chunk / tile machinery.
//
// With factor = false the stored factors and panel permutations are
// replayed on the right-hand columns only (used by iterative refinement).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hps_internal.cuh"
#include "tc_gemm.cuh"

namespace hps {
namespace lu {

constexpr int NT = 128;
constexpr int NWARP = NT / 32;

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int N = 2; };

template <typename T, int NB_>
struct Cfg {
    static constexpr int NB = NB_;
    static constexpr int HV = Vec<T>::N;   // elements per 16-byte vector
    // thread grid of the update tile: FP32 8 x 16 (64-row passes over
    // 128-column chunks, so a right-hand block of up to 128 columns is one
    // chunk), FP64 16 x 8 (64 x 32)
    static constexpr int TY = sizeof(T) == 4 ? 8 : 16, TX = NT / TY;
    static constexpr int CH = 2 * TX * HV;  // columns per chunk
};

// Shared-memory carve-up for one CTA.
template <typename T>
struct Smem {
    T *Ps;     // NB x ldp, panel (column-major)
    T *Us;     // NB x CH, current row block of the right part
    T *redv;   // NB + 8 + NWARP: argmax partials, sub-panel pivot row, diagonal reciprocals
    int *redi; // NWARP
    int *piv;  // NB: panel-relative pivot rows
    int *xsrc; // NB: source of displaced row j (or -1)
    int *xdst; // NB
    int *misc; // scalars: [0] leaf, [1] info, [2..] free
    int *map;  // ldp: row permutation scratch
    T *Ts;     // NB x NB: L11^-1 with its zeros and unit diagonal (FP32 path only)
};

// Whether an elimination keeps the inverses of its unit-lower diagonal blocks (FP32
// CUDA-core path with panels of 16 or 32 columns; see panel_inverses).
template <typename T, int NB, int TCK>
__host__ __device__ constexpr bool use_inverses() { return sizeof(T) == 4 && NB >= 16 && TCK == 0; }

template <typename T, int NB>
__host__ __device__ constexpr size_t smem_bytes_for(int ldp, bool with_ts = false) {
    return sizeof(T) * ((size_t)NB * ldp + (size_t)NB * Cfg<T, NB>::CH + NB + 8 + NWARP) +
           sizeof(int) * (NWARP + 3 * NB + 16 + ldp) + 64 + (with_ts ? sizeof(T) * NB * NB + 16 : 0);
}

template <typename T, int NB>
__device__ Smem<T> carve(unsigned char *base, int ldp) {
    Smem<T> s;
    T *t = (T *)base;
    s.Ps = t;
    t += (size_t)NB * ldp;
    s.Us = t;
    t += (size_t)NB * Cfg<T, NB>::CH;
    s.redv = t;
    t += NB + 8 + NWARP;
    int *ip = (int *)t;
    s.redi = ip;
    ip += NWARP;
    s.piv = ip;
    ip += NB;
    s.xsrc = ip;
    ip += NB;
    s.xdst = ip;
    ip += NB;
    s.misc = ip;
    ip += 16;
    s.map = ip;
    ip += ldp;
    s.Ts = (T *)(((uintptr_t)ip + 15) & ~(uintptr_t)15);
    return s;
}

template <typename T>
__device__ __forceinline__ T absval(T v) { return v < T(0) ? -v : v; }

// Asynchronous global -> shared copies (cp.async): every thread issues its
// copies without waiting on each load; cp_async_wait() then waits for this
// thread's copies, and a __syncthreads() publishes them to the CTA.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *s, const void *g) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    if constexpr (BYTES == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(g), "n"(BYTES) : "memory");
    }
}

__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Copy rows [0, rows) x columns [0, cols) of a row-major global block (ld
// LDC) to / from a column-major shared block (ld ldp).  Each warp touches
// whole 32-byte sectors of RW rows; with ldp = 4 (mod 32) the shared-memory
// side is free of bank conflicts for 4-byte elements.
template <typename T, bool TO_SHARED>
__device__ __forceinline__ void stage(T *__restrict__ g, int LDC, T *__restrict__ s, int ldp, int rows, int cols) {
    constexpr int SC = 32 / (int)sizeof(T);  // columns per sector
    constexpr int RW = 32 / SC;               // rows per warp instruction
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cin = lane % SC, rin = lane / SC;
    for (int cg = 0; cg < cols; cg += SC) {
        const int cc = cg + cin;
        if (cc >= cols) continue;
        for (int rg = warp * RW; rg < rows; rg += NWARP * RW) {
            const int rr = rg + rin;
            if (rr >= rows) continue;
            if (TO_SHARED) cp_async<sizeof(T)>(&s[cc * ldp + rr], &g[(long long)rr * LDC + cc]);
            else g[(long long)rr * LDC + cc] = s[cc * ldp + rr];
        }
    }
    if (TO_SHARED) cp_async_wait();
}

// Sub-panel width and the most panel rows a thread holds in registers.
template <typename T> struct PanelCfg;
template <> struct PanelCfg<float> { static constexpr int W = 8, RMAX = 8; };
template <> struct PanelCfg<double> { static constexpr int W = 8, RMAX = 4; };

// Magnitude key for the pivot search: |x| itself for float; for double the
// bit pattern with the sign cleared (non-negative IEEE doubles order like
// their bit patterns), so the comparisons stay off the FP64 pipe.  NaN keys
// order above every finite value.
template <typename T> struct MagKey;
template <> struct MagKey<float> {
    using K = float;
    __device__ static K of(float x) { return fabsf(x); }
    __device__ static K none() { return -1.0f; }
};
template <> struct MagKey<double> {
    using K = long long;
    __device__ static K of(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffLL; }
    __device__ static K none() { return -1LL; }
};

// Argmax of |value| over the CTA: (best, row) partials per thread -> the
// row index every thread agrees on (largest magnitude, first row on ties).
template <typename T>
__device__ __forceinline__ int block_argmax(typename MagKey<T>::K best, int bi, const Smem<T> &sm) {
    using K = typename MagKey<T>::K;
    K *redk = (K *)sm.redv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const K ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { redk[warp] = best; sm.redi[warp] = bi; }
    __syncthreads();
    best = redk[0];
    bi = sm.redi[0];
#pragma unroll
    for (int w = 1; w < NWARP; ++w) {
        const K ov = redk[w];
        const int oi = sm.redi[w];
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    return bi;
}

// Record pivot j -> pr (thread 0) in piv and the row map.
template <typename T>
__device__ __forceinline__ void record_pivot(int j, int pr, const Smem<T> &sm) {
    if (threadIdx.x == 0) {
        sm.piv[j] = pr;
        const int t = sm.map[j];
        sm.map[j] = sm.map[pr];
        sm.map[pr] = t;
    }
}

// Factor the shared-memory panel P (mp rows, nbk columns, ld ldp) with
// partial pivoting.  Also tracks the net row permutation in sm.map
// (panel-relative: row j of the factored panel is original row map[j]);
// sm.map must hold the identity on entry.  The first exact zero pivot sets
// sm.misc[1] (1-based, offset k0) and leaves its column unscaled.
//
// Sub-panels of W columns are factored with each thread holding its rows
// of the sub-panel in registers (rank-1 updates are register FMAs; row
// interchanges go through a small shared buffer); the rest of the panel is
// then updated as a block with the sub-panel's L still in registers.
// Panels taller than RMAX * NT rows use the shared-memory form throughout.
// Register form for panels of at most R * NT rows (R rows a thread).
template <typename T, int NB, int R>
__device__ void panel_factor_reg(T *__restrict__ P, int ldp, int mp, int nbk, int k0, const Smem<T> &sm);

template <typename T, int NB>
__device__ void panel_factor(T *__restrict__ P, int ldp, int mp, int nbk, int k0, const Smem<T> &sm) {
    constexpr int RMAX = PanelCfg<T>::RMAX;
    const int tid = threadIdx.x;
    if (mp > RMAX * NT) {
        for (int j = 0; j < nbk; ++j) {
            typename MagKey<T>::K best = MagKey<T>::none();
            int bi = 0x7fffffff;
            for (int i = j + tid; i < mp; i += NT) {
                const auto v = MagKey<T>::of(P[j * ldp + i]);
                if (v > best) { best = v; bi = i; }
            }
            bi = block_argmax<T>(best, bi, sm);
            const int pr = (bi >= mp || bi < j) ? j : bi;
            record_pivot<T>(j, pr, sm);
            if (pr != j) {
                for (int c = tid; c < nbk; c += NT) {
                    const T a = P[c * ldp + j];
                    P[c * ldp + j] = P[c * ldp + pr];
                    P[c * ldp + pr] = a;
                }
            }
            __syncthreads();
            const T pv = P[j * ldp + j];
            if (pv == T(0)) {
                if (tid == 0 && sm.misc[1] == 0) sm.misc[1] = k0 + j + 1;
            } else {
                const T inv = T(1) / pv;
                for (int i = j + 1 + tid; i < mp; i += NT) {
                    const T l = P[j * ldp + i] * inv;
                    P[j * ldp + i] = l;
#pragma unroll
                    for (int c = 1; c < NB; ++c)
                        if (c > j && c < nbk) P[c * ldp + i] = fma(-l, P[c * ldp + j], P[c * ldp + i]);
                }
            }
            __syncthreads();
        }
        return;
    }
    // the fewest register rows a thread needs for this panel's height
    if (mp <= NT) panel_factor_reg<T, NB, 1>(P, ldp, mp, nbk, k0, sm);
    else if (mp <= 2 * NT) panel_factor_reg<T, NB, 2>(P, ldp, mp, nbk, k0, sm);
    else if (mp <= 3 * NT) panel_factor_reg<T, NB, 3>(P, ldp, mp, nbk, k0, sm);
    else if (mp <= 4 * NT) panel_factor_reg<T, NB, 4>(P, ldp, mp, nbk, k0, sm);
    else if constexpr (RMAX > 4) panel_factor_reg<T, NB, RMAX>(P, ldp, mp, nbk, k0, sm);
}

template <typename T, int NB, int RMAX>
__device__ void panel_factor_reg(T *__restrict__ P, int ldp, int mp, int nbk, int k0, const Smem<T> &sm) {
    constexpr int W = PanelCfg<T>::W;
    using V = typename Vec<T>::type;
    constexpr int HV = Vec<T>::N;
    const int tid = threadIdx.x;
    T *bufA = sm.redv + NWARP;   // pivot row of the sub-panel (W values)
    T *bufB = sm.Us;             // displaced row (W values); Us is idle here
    for (int s0 = 0; s0 < nbk; s0 += W) {
        const int w = min(W, nbk - s0);
        // rows i = s0 + tid + t * NT of columns s0 .. s0 + w - 1 into registers
        T a[RMAX][W];
#pragma unroll
        for (int t = 0; t < RMAX; ++t) {
            const int i = s0 + tid + t * NT;
#pragma unroll
            for (int c = 0; c < W; ++c) a[t][c] = (i < mp && c < w) ? P[(s0 + c) * ldp + i] : T(0);
        }
#pragma unroll
        for (int jj = 0; jj < W; ++jj) {
            if (jj < w) {
                const int j = s0 + jj;
                typename MagKey<T>::K best = MagKey<T>::none();
                int bi = 0x7fffffff;
#pragma unroll
                for (int t = 0; t < RMAX; ++t) {
                    const int i = s0 + tid + t * NT;
                    const auto v = MagKey<T>::of(a[t][jj]);
                    if (i >= j && i < mp && v > best) { best = v; bi = i; }
                }
                bi = block_argmax<T>(best, bi, sm);
                const int pr = (bi >= mp || bi < j) ? j : bi;
                record_pivot<T>(j, pr, sm);
                // owners: row x belongs to thread (x - s0) % NT, slot (x - s0) / NT
                const int oj = (j - s0) % NT, sj = (j - s0) / NT;
                const int op = (pr - s0) % NT, sp = (pr - s0) / NT;
#pragma unroll
                for (int t = 0; t < RMAX; ++t) {
                    if (tid == op && t == sp)
#pragma unroll
                        for (int c = 0; c < W; ++c) bufA[c] = a[t][c];
                    if (pr != j && tid == oj && t == sj)
#pragma unroll
                        for (int c = 0; c < W; ++c) bufB[c] = a[t][c];
                }
                if (pr != j) {   // the panel columns outside the sub-panel
                    for (int c = tid; c < nbk; c += NT) {
                        if (c >= s0 && c < s0 + w) continue;
                        const T x = P[c * ldp + j];
                        P[c * ldp + j] = P[c * ldp + pr];
                        P[c * ldp + pr] = x;
                    }
                }
                __syncthreads();
                T prow[W];
#pragma unroll
                for (int c = 0; c < W; ++c) prow[c] = bufA[c];
                if (pr != j) {
#pragma unroll
                    for (int t = 0; t < RMAX; ++t) {
                        if (tid == oj && t == sj)
#pragma unroll
                            for (int c = 0; c < W; ++c) a[t][c] = prow[c];
                        if (tid == op && t == sp)
#pragma unroll
                            for (int c = 0; c < W; ++c) a[t][c] = bufB[c];
                    }
                }
                const T pv = prow[jj];
                if (pv == T(0)) {
                    if (tid == 0 && sm.misc[1] == 0) sm.misc[1] = k0 + j + 1;
                } else {
                    const T inv = T(1) / pv;
#pragma unroll
                    for (int t = 0; t < RMAX; ++t) {
                        const int i = s0 + tid + t * NT;
                        if (i > j && i < mp) {
                            const T l = a[t][jj] * inv;
                            a[t][jj] = l;
#pragma unroll
                            for (int c = jj + 1; c < W; ++c) a[t][c] = fma(-l, prow[c], a[t][c]);
                        }
                    }
                }
            }
        }
        // sub-panel back to shared memory
#pragma unroll
        for (int t = 0; t < RMAX; ++t) {
            const int i = s0 + tid + t * NT;
            if (i < mp)
#pragma unroll
                for (int c = 0; c < W; ++c)
                    if (c < w) P[(s0 + c) * ldp + i] = a[t][c];
        }
        __syncthreads();
        if (s0 + w < nbk) {
            // top rows of the remaining columns: U = L11^{-1} A (unit lower)
            for (int c = s0 + w + tid; c < nbk; c += NT) {
                T u[W];
#pragma unroll
                for (int k = 0; k < W; ++k) u[k] = P[c * ldp + s0 + k];
#pragma unroll
                for (int k = 0; k < W; ++k)
#pragma unroll
                    for (int i2 = k + 1; i2 < W; ++i2) u[i2] = fma(-P[(s0 + k) * ldp + s0 + i2], u[k], u[i2]);
#pragma unroll
                for (int k = 0; k < W; ++k) P[c * ldp + s0 + k] = u[k];
            }
            __syncthreads();
            // rows below: A -= L (registers) * U (shared, 16-byte loads)
            for (int c = s0 + w; c < nbk; ++c) {
                T u[W];
#pragma unroll
                for (int g = 0; g < W / HV; ++g) {
                    const V uv = *(const V *)(P + c * ldp + s0 + g * HV);
                    const T *pu = (const T *)&uv;
#pragma unroll
                    for (int t = 0; t < HV; ++t) u[g * HV + t] = pu[t];
                }
#pragma unroll
                for (int t = 0; t < RMAX; ++t) {
                    const int i = s0 + tid + t * NT;
                    if (i >= s0 + w && i < mp) {
                        T v = P[c * ldp + i];
#pragma unroll
                        for (int k = 0; k < W; ++k) v = fma(-a[t][k], u[k], v);
                        P[c * ldp + i] = v;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Net row permutation of the panel's interchanges (panel-relative rows),
// from the pivots and the map left by panel_factor: top row j receives
// source map[j]; displaced rows below the panel receive xsrc[j] at xdst[j]
// (xdst = -1 when nothing lands there from step j).  The sources of
// displaced rows are always top rows, so gathering every source before any
// store is race-free.
template <typename T>
__device__ void panel_permutation(int nbk, const Smem<T> &sm) {
    const int tid = threadIdx.x;
    for (int j = tid; j < nbk; j += NT) {
        const int p = sm.piv[j];
        bool last = p >= nbk;
        for (int j2 = j + 1; j2 < nbk && last; ++j2) last = sm.piv[j2] != p;
        sm.xdst[j] = last ? p : -1;
        sm.xsrc[j] = last ? sm.map[p] : -1;
    }
    __syncthreads();
}

// Inverse of the unit-lower diagonal block of a factored panel (FP32 path).
// The top nbk x nbk block of the shared panel P holds L11 below its
// diagonal; it is replaced in place by L11^-1 (also unit lower), which then
// travels to the workspace with the panel.  The U12 rows of every update
// chunk, in the factorization and in the refinement replays, are then one
// product whose outputs are independent dot products (tri_mul) instead of
// a chain of nbk dependent steps per column.  With partial pivoting
// |L11| <= 1 and its inverse stays well scaled; U11, which carries the
// conditioning of the leaf, keeps its substitution in the back solve.
// Warp 0 forms column j of L11^-1 (thread j) by substitution on e_j; Ts
// receives the inverse with its unit diagonal and zeros written out.
template <typename T, int NB>
__device__ void panel_inverses(T *__restrict__ P, int ldp, int nbk, const Smem<T> &sm) {
    using V = typename Vec<T>::type;
    constexpr int HV = Vec<T>::N;
    static_assert(NB <= 32, "one warp of NB columns");
    const int j = threadIdx.x;
    T x[NB];
    if (j < NB) {
#pragma unroll
        for (int i = 0; i < NB; ++i) x[i] = i == j ? T(1) : T(0);
        // forward: after step k, x[k + 1] is final (x[i < j] stay 0)
#pragma unroll
        for (int k = 0; k < NB - 1; ++k) {
            const T xk = x[k];
            const T *col = P + k * ldp;
#pragma unroll
            for (int g = (k + 1) / HV; g < NB / HV; ++g) {
                const V lv = *(const V *)(col + g * HV);
                const T *pl = (const T *)&lv;
#pragma unroll
                for (int t = 0; t < HV; ++t)
                    if (g * HV + t > k) x[g * HV + t] = fma(-pl[t], xk, x[g * HV + t]);
            }
        }
    }
    __syncthreads();
    if (j < NB) {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            if (i > j && i < nbk) P[j * ldp + i] = x[i];
            sm.Ts[j * NB + i] = (i < nbk && j < nbk) ? x[i] : T(0);
        }
    }
    __syncthreads();
}

// Rows [0, nbk) x columns [0, cw) of the chunk Us replaced by Ts * Us and
// also written to rows row0.. (columns c0..) of M.  Ts is NB x NB
// column-major with its zeros present, so each output is one dot product.
// Thread tile: 4 rows x NB/4 columns (NB/16 vectors of 4, spread so a
// warp's vector loads of Us are consecutive).
template <typename T, int NB>
__device__ void tri_mul(const Smem<T> &sm, int nbk, int cw, T *__restrict__ M, int LDC, int row0, int c0) {
    static_assert(sizeof(T) == 4 && NB >= 16, "FP32 path, panels of 16 or 32");
    constexpr int CH = Cfg<T, NB>::CH, RG = NB / 4, TXC = NT / RG, NV = CH / (4 * TXC);
    const int tx = threadIdx.x % TXC, ty = threadIdx.x / TXC;
    float acc[4][4 * NV];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4 * NV; ++v) acc[u][v] = 0.0f;
#pragma unroll 4
    for (int k = 0; k < nbk; ++k) {
        const float4 a = *(const float4 *)(sm.Ts + k * NB + ty * 4);
        const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const float4 b = *(const float4 *)(sm.Us + k * CH + v * 4 * TXC + tx * 4);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc[u][4 * v] = fmaf(av[u], b.x, acc[u][4 * v]);
                acc[u][4 * v + 1] = fmaf(av[u], b.y, acc[u][4 * v + 1]);
                acc[u][4 * v + 2] = fmaf(av[u], b.z, acc[u][4 * v + 2]);
                acc[u][4 * v + 3] = fmaf(av[u], b.w, acc[u][4 * v + 3]);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = ty * 4 + u;
        if (i >= nbk) continue;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int c = v * 4 * TXC + tx * 4;
            if (c >= cw) continue;   // a vector that starts inside cw may end in the row padding
            const float4 o = make_float4(acc[u][4 * v], acc[u][4 * v + 1], acc[u][4 * v + 2], acc[u][4 * v + 3]);
            *(float4 *)(sm.Us + i * CH + c) = o;
            *(float4 *)(M + (long long)(row0 + i) * LDC + c0 + c) = o;
        }
    }
}

// Mg[r, c0 + c] -= sum_kk A[kk*lda + r - arow0] * B[kk*CH + c] for rows
// [r0, r1), columns [0, cw).  A and B in shared memory.
template <typename T, int NB>
__device__ __forceinline__ void gemm_sub(T *__restrict__ Mg, int LDC, int r0, int r1, int c0, int cw,
                                         const T *__restrict__ A, int lda, int arow0,
                                         const T *__restrict__ B, int K) {
    using CF = Cfg<T, NB>;
    using V = typename Vec<T>::type;
    constexpr int HV = CF::HV, TX = CF::TX, CH = CF::CH;
    // threads across the columns: just enough 2HV-column tiles for cw (a
    // full chunk uses TX of them); the rest of the CTA goes to rows
    const int txr = min(TX, (cw + 2 * HV - 1) / (2 * HV)), tyr = NT / txr;
    if (threadIdx.x >= txr * tyr) return;
    const int tx = threadIdx.x % txr, ty = threadIdx.x / txr;
    const int cA = tx * HV, cB = txr * HV + tx * HV;
    for (int rb = r0; rb < r1; rb += 2 * tyr * HV) {
        int sa = rb + ty * HV, sb = rb + tyr * HV + ty * HV;
        const bool va = sa < r1, vb = sb < r1;
        if (!va && !vb) continue;
        const int ia = (va ? sa : r0) - arow0, ib = (vb ? sb : r0) - arow0;
        // FP64: accumulate straight into the loaded C tile (C -= a b per
        // step), so the FP64 pipe carries no separate subtraction; FP32:
        // accumulate the product from zero and subtract once (C - sum ab
        // keeps the FP32 factors measurably more accurate).
        constexpr bool INPLACE = sizeof(T) == 8;
        T acc[2 * HV][2 * HV];
#pragma unroll
        for (int u = 0; u < 2 * HV; ++u)
#pragma unroll
            for (int v = 0; v < 2 * HV; ++v) acc[u][v] = T(0);
        if constexpr (INPLACE) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int s = half ? sb : sa;
#pragma unroll
                for (int u = 0; u < HV; ++u) {
                    const T *row = Mg + (long long)min(s + u, r1 - 1) * LDC + c0;
#pragma unroll
                    for (int hc = 0; hc < 2; ++hc) {
                        const int c = hc ? cB : cA;
                        const V cv = *(const V *)(row + (c < cw ? c : 0));
                        const T *pc = (const T *)&cv;
#pragma unroll
                        for (int v = 0; v < HV; ++v) acc[half * HV + u][hc * HV + v] = pc[v];
                    }
                }
            }
        }
        const T sgn = INPLACE ? T(-1) : T(1);
#pragma unroll 4
        for (int kk = 0; kk < K; ++kk) {
            const V a0 = *(const V *)(A + kk * lda + ia);
            const V a1 = *(const V *)(A + kk * lda + ib);
            const V b0 = *(const V *)(B + kk * CH + cA);
            const V b1 = *(const V *)(B + kk * CH + cB);
            const T *pa0 = (const T *)&a0, *pa1 = (const T *)&a1;
            const T *pb0 = (const T *)&b0, *pb1 = (const T *)&b1;
#pragma unroll
            for (int u = 0; u < HV; ++u) {
                const T x0 = sgn * pa0[u], x1 = sgn * pa1[u];
#pragma unroll
                for (int v = 0; v < HV; ++v) {
                    acc[u][v] = fma(x0, pb0[v], acc[u][v]);
                    acc[u][HV + v] = fma(x0, pb1[v], acc[u][HV + v]);
                    acc[HV + u][v] = fma(x1, pb0[v], acc[HV + u][v]);
                    acc[HV + u][HV + v] = fma(x1, pb1[v], acc[HV + u][HV + v]);
                }
            }
        }
        if constexpr (INPLACE) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int s = half ? sb : sa;
#pragma unroll
                for (int u = 0; u < HV; ++u) {
                    const int r = s + u;
                    if (r >= r1) continue;
                    T *row = Mg + (long long)r * LDC + c0;
#pragma unroll
                    for (int hc = 0; hc < 2; ++hc) {
                        const int c = hc ? cB : cA;
                        if (c >= cw) continue;
                        V cv;
                        T *pc = (T *)&cv;
#pragma unroll
                        for (int v = 0; v < HV; ++v) pc[v] = acc[half * HV + u][hc * HV + v];
                        *(V *)(row + c) = cv;
                    }
                }
            }
            continue;
        }
        // C -= acc, one half of the rows at a time: the half's 2HV vector
        // loads are all issued before the first subtraction
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int s = half ? sb : sa;
            V cv[HV][2];
#pragma unroll
            for (int u = 0; u < HV; ++u) {
                const int r = min(s + u, r1 - 1);
                const T *row = Mg + (long long)r * LDC + c0;
#pragma unroll
                for (int hc = 0; hc < 2; ++hc) {
                    const int c = hc ? cB : cA;
                    cv[u][hc] = *(const V *)(row + (c < cw ? c : 0));   // clamped: stays in the row
                }
            }
#pragma unroll
            for (int u = 0; u < HV; ++u) {
                const int r = s + u;
                if (r >= r1) continue;
                T *row = Mg + (long long)r * LDC + c0;
#pragma unroll
                for (int hc = 0; hc < 2; ++hc) {
                    const int c = hc ? cB : cA;
                    if (c >= cw) continue;
                    T *pc = (T *)&cv[u][hc];
#pragma unroll
                    for (int v = 0; v < HV; ++v) pc[v] -= acc[half * HV + u][hc * HV + v];
                    *(V *)(row + c) = cv[u][hc];
                }
            }
        }
    }
}

// C[r0:r1, c0:c0+cw] -= A * B on the tensor cores (see tc_gemm.cuh): A from
// the shared panel (column-major, ld lda, rows offset arow0), B = the shared
// chunk (K x CH, row-major), K <= NB (zero-padded to NB).
template <int KIND, int NB>
__device__ void gemm_sub_tc(float *__restrict__ Mg, int LDC, int r0, int r1, int c0, int cw,
                            const float *__restrict__ A, int lda, int arow0, const float *__restrict__ B, int K,
                            const tc::TcState &ts) {
    using namespace tc;
    constexpr int EB = In<KIND>::BYTES, PER = 16 / EB, KS = In<KIND>::KSTEP;
    constexpr int CH = Cfg<float, NB>::CH;
    static_assert(CH % TN == 0, "chunk width must be a multiple of the MMA tile width");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int cb = 0; cb < cw; cb += TN) {
    const int cwh = min(TN, cw - cb);
    // B (the chunk's U12 rows, as TN x NB K-major): element (c, k) = B[k][c]
    for (int e = tid; e < TN * (NB / PER); e += NT) {   // one core-matrix row (PER k) per thread
        const int c = e % TN, g = e / TN;
        float x[PER];
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int k = g * PER + t;
            x[t] = (k < K && c < cwh) ? B[k * CH + cb + c] : 0.0f;
        }
        const int off = kmajor_off<KIND>(c, g * PER, NB);
        SplitRow<KIND>::store(ts.b_hi + off, ts.b_lo + off, x);
    }
    const uint32_t idesc = instr_desc<KIND>();
    const uint32_t lbo = 128, sbo = (NB / PER) * 128;
    for (int rb = r0; rb < r1; rb += TM) {
        for (int e = tid; e < TM * (NB / PER); e += NT) {
            const int r = e % TM, g = e / TM, row = rb + r;
            float x[PER];
#pragma unroll
            for (int t = 0; t < PER; ++t) {
                const int k = g * PER + t;
                x[t] = (row < r1 && k < K) ? A[k * lda + (row - arow0)] : 0.0f;
            }
            const int off = kmajor_off<KIND>(r, g * PER, NB);
            SplitRow<KIND>::store(ts.a_hi + off, ts.a_lo + off, x);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t tmem = *ts.tmem, phase = *ts.phase;
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < NB / KS; ++ks) {
                const uint32_t step = ks * (KS / PER) * 128;
                const uint64_t ah = smem_desc(smem_addr(ts.a_hi) + step, lbo, sbo);
                const uint64_t al = smem_desc(smem_addr(ts.a_lo) + step, lbo, sbo);
                const uint64_t bh = smem_desc(smem_addr(ts.b_hi) + step, lbo, sbo);
                const uint64_t bl = smem_desc(smem_addr(ts.b_lo) + step, lbo, sbo);
                mma(tmem, ah, bh, idesc, ks > 0, KIND);
                mma(tmem, ah, bl, idesc, 1, KIND);
                mma(tmem, al, bh, idesc, 1, KIND);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_addr(ts.mbar)));
        }
        const bool ok = __all_sync(0xffffffffu, wait_mma(ts, phase));
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (ok) {
            const int row = rb + warp * 32 + lane;
            float *crow = Mg + (long long)min(row, r1 - 1) * LDC + c0 + cb;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float v[32];
                ld_row32(tmem + ((uint32_t)(warp * 32) << 16) + half * 32, v);
                if (row < r1) {
#pragma unroll
                    for (int g = 0; g < 8; ++g) {
                        const int c = half * 32 + g * 4;
                        if (c < cwh) {
                            float4 cv = *(float4 *)(crow + c);
                            cv.x -= v[g * 4];
                            cv.y -= v[g * 4 + 1];
                            cv.z -= v[g * 4 + 2];
                            cv.w -= v[g * 4 + 3];
                            *(float4 *)(crow + c) = cv;
                        }
                    }
                }
            }
        } else if (lane == 0) {
            atomicExch(ts.err, 1);
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (tid == 0) *ts.phase = phase ^ 1u;
    }
    }
}

// Apply the panel at rows k0.. (permutation, unit-lower solve, trailing
// update) to columns [cstart, C) of M.
template <typename T, int NB, int TCK = 0, bool INV = false>
__device__ void apply_panel(T *__restrict__ M, int LDC, int n, int C, int k0, int nbk, int cstart, int ldp,
                            const Smem<T> &sm, const tc::TcState *ts = nullptr) {
    using CF = Cfg<T, NB>;
    using V = typename Vec<T>::type;
    constexpr int CH = CF::CH, HV = CF::HV;
    constexpr int XPT = (NB * CH + NT - 1) / NT;  // displaced-row elements per thread
    const int tid = threadIdx.x;
    for (int c0 = cstart; c0 < C; c0 += CH) {
        const int cw = min(CH, C - c0);
        // gather: top rows into Us (16-byte asynchronous copies; a vector
        // starting before cw ends inside the padded row), displaced rows
        // into registers
        constexpr int VPR = CH / HV;
        for (int e = tid; e < nbk * VPR; e += NT) {
            const int j = e / VPR, c = (e % VPR) * HV;
            if (c < cw) cp_async<16>(&sm.Us[j * CH + c], &M[(long long)(k0 + sm.map[j]) * LDC + c0 + c]);
        }
        T xv[XPT];
#pragma unroll
        for (int t = 0; t < XPT; ++t) {
            const int e = tid + t * NT;
            const int j = e / CH, c = e % CH;
            xv[t] = T(0);
            if (e < nbk * CH && c < cw && sm.xsrc[j] >= 0) xv[t] = M[(long long)(k0 + sm.xsrc[j]) * LDC + c0 + c];
        }
        cp_async_wait();
        __syncthreads();
#pragma unroll
        for (int t = 0; t < XPT; ++t) {
            const int e = tid + t * NT;
            const int j = e / CH, c = e % CH;
            if (e < nbk * CH && c < cw && sm.xdst[j] >= 0) M[(long long)(k0 + sm.xdst[j]) * LDC + c0 + c] = xv[t];
        }
        // unit-lower solve: with the inverse kept in Ts, one product;
        // otherwise one column per thread, column in registers,
        // column-oriented (axpy) so each step's multipliers L[j+1.., j] are
        // consecutive in the shared panel and load as 16-byte vectors
        if constexpr (INV) tri_mul<T, NB>(sm, nbk, cw, M, LDC, k0, c0);
        else for (int c = tid; c < cw; c += NT) {
            T u[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) u[j] = j < nbk ? sm.Us[j * CH + c] : T(0);
#pragma unroll
            for (int j = 0; j < NB - 1; ++j) {
                if (j < nbk) {
                    const T uj = u[j];
                    const T *col = sm.Ps + j * ldp;
#pragma unroll
                    for (int g = (j + 1) / HV; g < NB / HV; ++g) {
                        const V lv = *(const V *)(col + g * HV);
                        const T *pl = (const T *)&lv;
#pragma unroll
                        for (int t = 0; t < HV; ++t)
                            if (g * HV + t > j) u[g * HV + t] = fma(-pl[t], uj, u[g * HV + t]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                if (j < nbk) {
                    sm.Us[j * CH + c] = u[j];
                    M[(long long)(k0 + j) * LDC + c0 + c] = u[j];
                }
            }
        }
        __syncthreads();
        if constexpr (TCK != 0) {
            if (ts) gemm_sub_tc<TCK, NB>(M, LDC, k0 + nbk, n, c0, cw, sm.Ps, ldp, k0, sm.Us, nbk, *ts);
            else gemm_sub<T, NB>(M, LDC, k0 + nbk, n, c0, cw, sm.Ps, ldp, k0, sm.Us, nbk);
        } else {
            gemm_sub<T, NB>(M, LDC, k0 + nbk, n, c0, cw, sm.Ps, ldp, k0, sm.Us, nbk);
        }
        __syncthreads();
    }
}

// Elimination on M = [A (n cols) | pad | RHS from column n4], C columns in
// all, row-major with ld LDC (multiple of 4; M 16-byte aligned).  When
// perm_g is given, factoring stores each panel's permutation there (3 NB
// ints per panel: top-row sources, displaced sources, displaced targets)
// and replaying (factor = false) reads it back.
template <typename T, int NB, int TCK = 0, bool INV = false>
__device__ void lu_solve(T *__restrict__ M, int LDC, int n, int n4, int C, bool factor, int *perm_g, int ldp,
                         const Smem<T> &sm, const tc::TcState *ts = nullptr) {
    using CF = Cfg<T, NB>;
    using V = typename Vec<T>::type;
    constexpr int CH = CF::CH, HV = CF::HV;
    const int tid = threadIdx.x;
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int nbk = min(NB, n - k0), mp = n - k0;
        int *pg = perm_g ? perm_g + 3 * k0 : nullptr;
        if (factor)
            for (int r = tid; r < mp; r += NT) sm.map[r] = r;
        else
            for (int j = tid; j < nbk; j += NT) {
                sm.map[j] = pg[j];
                sm.xsrc[j] = pg[NB + j];
                sm.xdst[j] = pg[2 * NB + j];
            }
        stage<T, true>(M + (long long)k0 * LDC + k0, LDC, sm.Ps, ldp, mp, nbk);
        __syncthreads();
        if constexpr (INV) {
            if (!factor) {   // L11^-1 from the stored panel, zeros and unit diagonal written out
                for (int e = tid; e < NB * NB; e += NT) {
                    const int k = e / NB, i = e - k * NB;
                    sm.Ts[e] = (i < nbk && k < nbk) ? (i > k ? sm.Ps[k * ldp + i] : (i == k ? T(1) : T(0))) : T(0);
                }
                __syncthreads();
            }
        }
        if (factor) {
            panel_factor<T, NB>(sm.Ps, ldp, mp, nbk, k0, sm);
            if constexpr (INV) panel_inverses<T, NB>(sm.Ps, ldp, nbk, sm);
            stage<T, false>(M + (long long)k0 * LDC + k0, LDC, sm.Ps, ldp, mp, nbk);
            panel_permutation<T>(nbk, sm);
            if (pg)
                for (int j = tid; j < nbk; j += NT) {
                    pg[j] = sm.map[j];
                    pg[NB + j] = sm.xsrc[j];
                    pg[2 * NB + j] = sm.xdst[j];
                }
        }
        const int cstart = factor ? (k0 + nbk < n ? k0 + nbk : n4) : n4;
        // the factorization's trailing updates go to the tensor cores when
        // enabled; the right-hand-only replays stay on the FP32 pipe
        apply_panel<T, NB, TCK, INV>(M, LDC, n, C, k0, nbk, cstart, ldp, sm, factor ? ts : nullptr);
    }

    // U X = Y for the right-hand columns, block rows from the bottom
    for (int kb0 = ((n - 1) / NB) * NB; kb0 >= 0; kb0 -= NB) {
        const int nbk = min(NB, n - kb0), rows = kb0 + nbk;
        stage<T, true>(M + kb0, LDC, sm.Ps, ldp, rows, nbk);
        __syncthreads();
        for (int j = tid; j < nbk; j += NT) sm.redv[j] = T(1) / sm.Ps[j * ldp + kb0 + j];
        __syncthreads();
        for (int c0 = n4; c0 < C; c0 += CH) {
            const int cw = min(CH, C - c0);
            for (int c = tid; c < cw; c += NT) {
                T u[NB];
#pragma unroll
                for (int j = 0; j < NB; ++j) u[j] = j < nbk ? M[(long long)(kb0 + j) * LDC + c0 + c] : T(0);
                // column-oriented: u[i] /= U[i][i], then u[j] -= U[j][i] u[i]
                // for j < i, with U[0..i)[i] consecutive in the shared block
#pragma unroll
                for (int i = NB - 1; i >= 0; --i) {
                    if (i < nbk) {
                        const T *col = sm.Ps + i * ldp + kb0;
                        const T ui = u[i] * sm.redv[i];
                        u[i] = ui;
#pragma unroll
                        for (int g = 0; g < (i + HV - 1) / HV; ++g) {
                            const V uv = *(const V *)(col + g * HV);
                            const T *pu = (const T *)&uv;
#pragma unroll
                            for (int t = 0; t < HV; ++t)
                                if (g * HV + t < i) u[g * HV + t] = fma(-pu[t], ui, u[g * HV + t]);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    if (j < nbk) {
                        sm.Us[j * CH + c] = u[j];
                        M[(long long)(kb0 + j) * LDC + c0 + c] = u[j];
                    }
                }
            }
            __syncthreads();
            gemm_sub<T, NB>(M, LDC, 0, kb0, c0, cw, sm.Ps, ldp, 0, sm.Us, nbk);
            __syncthreads();
        }
    }
}

// Leading dimension of the shared panel: at least nmax + 8 rows (room for
// the straddle of one 16-byte vector past the last row), 4 (mod 32).
__host__ __device__ inline int panel_ld(int nmax) { return ((nmax + 4 + 31) / 32) * 32 + 4; }

}  // namespace lu
}  // namespace hps
