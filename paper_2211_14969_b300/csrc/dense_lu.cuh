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
// With factor = false the stored factors and pivots are replayed on the
// right-hand columns only (used by iterative refinement).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hps_internal.cuh"

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
    static constexpr int TY = 16, TX = 8;  // thread grid of the update tile
    static constexpr int BM = 2 * TY * HV;  // rows per update pass
    static constexpr int CH = 2 * TX * HV;  // columns per chunk
};

// Shared-memory carve-up for one CTA.
template <typename T>
struct Smem {
    T *Ps;     // NB x ldp, panel (column-major)
    T *Us;     // NB x CH, current row block of the right part
    T *redv;   // NWARP
    int *redi; // NWARP
    int *piv;  // NB: panel-relative pivot rows
    int *xsrc; // NB: source of displaced row j (or -1)
    int *xdst; // NB
    int *misc; // scalars: [0] leaf, [1] info, [2..] free
    int *map;  // ldp: row permutation scratch
};

template <typename T, int NB>
__host__ __device__ constexpr size_t smem_bytes_for(int ldp) {
    return sizeof(T) * ((size_t)NB * ldp + (size_t)NB * Cfg<T, NB>::CH + 2 * NWARP) +
           sizeof(int) * (NWARP + 3 * NB + 16 + ldp) + 64;
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
    t += 2 * NWARP;
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
    return s;
}

template <typename T>
__device__ __forceinline__ T absval(T v) { return v < T(0) ? -v : v; }

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
            if (TO_SHARED) s[cc * ldp + rr] = g[(long long)rr * LDC + cc];
            else g[(long long)rr * LDC + cc] = s[cc * ldp + rr];
        }
    }
}

// Factor the shared-memory panel P (mp rows, nbk columns, ld ldp).
template <typename T>
__device__ void panel_factor(T *__restrict__ P, int ldp, int mp, int nbk, int k0, const Smem<T> &sm) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = 0; j < nbk; ++j) {
        T best = T(-1);
        int bi = 0x7fffffff;
        for (int i = j + tid; i < mp; i += NT) {
            const T v = absval(P[j * ldp + i]);
            if (v > best) { best = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { sm.redv[warp] = best; sm.redi[warp] = bi; }
        __syncthreads();
        best = sm.redv[0];
        bi = sm.redi[0];
#pragma unroll
        for (int w = 1; w < NWARP; ++w) {
            const T ov = sm.redv[w];
            const int oi = sm.redi[w];
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        const int pr = (bi >= mp || bi < j) ? j : bi;   // no finite candidate: keep the row
        if (tid == 0) sm.piv[j] = pr;
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
                for (int c = j + 1; c < nbk; ++c) P[c * ldp + i] = fma(-l, P[c * ldp + j], P[c * ldp + i]);
            }
        }
        __syncthreads();
    }
}

// Net row permutation of the panel's interchanges (panel-relative rows):
// top row j receives source map[j]; displaced rows below the panel receive
// xsrc[j] at xdst[j] (xdst = -1 when nothing lands there from step j).
template <typename T>
__device__ void panel_permutation(int mp, int nbk, const Smem<T> &sm) {
    const int tid = threadIdx.x;
    for (int r = tid; r < mp; r += NT) sm.map[r] = r;
    __syncthreads();
    if (tid == 0) {
        for (int j = 0; j < nbk; ++j) {
            const int p = sm.piv[j];
            const int t = sm.map[j];
            sm.map[j] = sm.map[p];
            sm.map[p] = t;
        }
    }
    __syncthreads();
    for (int j = tid; j < nbk; j += NT) {
        const int p = sm.piv[j];
        bool last = p >= nbk;
        for (int j2 = j + 1; j2 < nbk && last; ++j2) last = sm.piv[j2] != p;
        sm.xdst[j] = last ? p : -1;
        sm.xsrc[j] = last ? sm.map[p] : -1;
    }
    __syncthreads();
}

// Mg[r, c0 + c] -= sum_kk A[kk*lda + r - arow0] * B[kk*CH + c] for rows
// [r0, r1), columns [0, cw).  A and B in shared memory.
template <typename T, int NB>
__device__ __forceinline__ void gemm_sub(T *__restrict__ Mg, int LDC, int r0, int r1, int c0, int cw,
                                         const T *__restrict__ A, int lda, int arow0,
                                         const T *__restrict__ B, int K) {
    using CF = Cfg<T, NB>;
    using V = typename Vec<T>::type;
    constexpr int HV = CF::HV, TY = CF::TY, TX = CF::TX, CH = CF::CH;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int cA = tx * HV, cB = TX * HV + tx * HV;
    for (int rb = r0; rb < r1; rb += CF::BM) {
        int sa = rb + ty * HV, sb = rb + TY * HV + ty * HV;
        const bool va = sa < r1, vb = sb < r1;
        if (!va && !vb) continue;
        const int ia = (va ? sa : r0) - arow0, ib = (vb ? sb : r0) - arow0;
        T acc[2 * HV][2 * HV];
#pragma unroll
        for (int u = 0; u < 2 * HV; ++u)
#pragma unroll
            for (int v = 0; v < 2 * HV; ++v) acc[u][v] = T(0);
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
#pragma unroll
                for (int v = 0; v < HV; ++v) {
                    acc[u][v] = fma(pa0[u], pb0[v], acc[u][v]);
                    acc[u][HV + v] = fma(pa0[u], pb1[v], acc[u][HV + v]);
                    acc[HV + u][v] = fma(pa1[u], pb0[v], acc[HV + u][v]);
                    acc[HV + u][HV + v] = fma(pa1[u], pb1[v], acc[HV + u][HV + v]);
                }
            }
        }
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
                    V cv = *(V *)(row + c);
                    T *pc = (T *)&cv;
#pragma unroll
                    for (int v = 0; v < HV; ++v) pc[v] -= acc[half * HV + u][hc * HV + v];
                    *(V *)(row + c) = cv;
                }
            }
        }
    }
}

// Apply the panel at rows k0.. (permutation, unit-lower solve, trailing
// update) to columns [cstart, C) of M.
template <typename T, int NB>
__device__ void apply_panel(T *__restrict__ M, int LDC, int n, int C, int k0, int nbk, int cstart, int ldp,
                            const Smem<T> &sm) {
    using CF = Cfg<T, NB>;
    constexpr int CH = CF::CH;
    constexpr int XPT = (NB * CH + NT - 1) / NT;  // displaced-row elements per thread
    const int tid = threadIdx.x;
    for (int c0 = cstart; c0 < C; c0 += CH) {
        const int cw = min(CH, C - c0);
        // gather: top rows into Us, displaced rows into registers
        for (int e = tid; e < nbk * CH; e += NT) {
            const int j = e / CH, c = e % CH;
            if (c < cw) sm.Us[j * CH + c] = M[(long long)(k0 + sm.map[j]) * LDC + c0 + c];
        }
        T xv[XPT];
#pragma unroll
        for (int t = 0; t < XPT; ++t) {
            const int e = tid + t * NT;
            const int j = e / CH, c = e % CH;
            xv[t] = T(0);
            if (e < nbk * CH && c < cw && sm.xsrc[j] >= 0) xv[t] = M[(long long)(k0 + sm.xsrc[j]) * LDC + c0 + c];
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < XPT; ++t) {
            const int e = tid + t * NT;
            const int j = e / CH, c = e % CH;
            if (e < nbk * CH && c < cw && sm.xdst[j] >= 0) M[(long long)(k0 + sm.xdst[j]) * LDC + c0 + c] = xv[t];
        }
        // unit-lower solve, one column per thread, column in registers
        for (int c = tid; c < cw; c += NT) {
            T u[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) u[j] = j < nbk ? sm.Us[j * CH + c] : T(0);
#pragma unroll
            for (int j = 1; j < NB; ++j) {
                if (j < nbk) {
                    T v = u[j];
#pragma unroll
                    for (int i = 0; i < j; ++i) v = fma(-sm.Ps[i * ldp + j], u[i], v);
                    u[j] = v;
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
        gemm_sub<T, NB>(M, LDC, k0 + nbk, n, c0, cw, sm.Ps, ldp, k0, sm.Us, nbk);
        __syncthreads();
    }
}

// Elimination on M = [A (n cols) | pad | RHS from column n4], C columns in
// all, row-major with ld LDC (multiple of 4; M 16-byte aligned).
template <typename T, int NB>
__device__ void lu_solve(T *__restrict__ M, int LDC, int n, int n4, int C, bool factor, int *piv_g, int ldp,
                         const Smem<T> &sm) {
    using CF = Cfg<T, NB>;
    constexpr int CH = CF::CH;
    const int tid = threadIdx.x;
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int nbk = min(NB, n - k0), mp = n - k0;
        stage<T, true>(M + (long long)k0 * LDC + k0, LDC, sm.Ps, ldp, mp, nbk);
        if (!factor)
            for (int j = tid; j < nbk; j += NT) sm.piv[j] = piv_g[k0 + j] - k0;
        __syncthreads();
        if (factor) {
            panel_factor<T>(sm.Ps, ldp, mp, nbk, k0, sm);
            stage<T, false>(M + (long long)k0 * LDC + k0, LDC, sm.Ps, ldp, mp, nbk);
            if (piv_g)
                for (int j = tid; j < nbk; j += NT) piv_g[k0 + j] = k0 + sm.piv[j];
        }
        panel_permutation<T>(mp, nbk, sm);
        const int cstart = factor ? (k0 + nbk < n ? k0 + nbk : n4) : n4;
        apply_panel<T, NB>(M, LDC, n, C, k0, nbk, cstart, ldp, sm);
    }

    // U X = Y for the right-hand columns, block rows from the bottom
    for (int kb0 = ((n - 1) / NB) * NB; kb0 >= 0; kb0 -= NB) {
        const int nbk = min(NB, n - kb0), rows = kb0 + nbk;
        stage<T, true>(M + kb0, LDC, sm.Ps, ldp, rows, nbk);
        __syncthreads();
        for (int c0 = n4; c0 < C; c0 += CH) {
            const int cw = min(CH, C - c0);
            for (int c = tid; c < cw; c += NT) {
                T u[NB];
#pragma unroll
                for (int j = 0; j < NB; ++j) u[j] = j < nbk ? M[(long long)(kb0 + j) * LDC + c0 + c] : T(0);
#pragma unroll
                for (int j = NB - 1; j >= 0; --j) {
                    if (j < nbk) {
                        T v = u[j];
#pragma unroll
                        for (int i = j + 1; i < NB; ++i)
                            if (i < nbk) v = fma(-sm.Ps[i * ldp + kb0 + j], u[i], v);
                        u[j] = v / sm.Ps[j * ldp + kb0 + j];
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
