// Blocked dense LU with partial pivoting on an augmented row-major matrix
// [A | RHS], run by one CTA of kThreads threads: the panel is factored in
// shared memory with a warp-shuffle pivot search, the row swaps and the
// unit-lower solve are applied to the right-hand columns in chunks staged in
// shared memory, and the trailing update is register-tiled.  Then U X = Y is
// solved in place for the right-hand columns.  Shared by the leaf
// condensation and the merge kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hps_internal.cuh"

namespace hps {
namespace lu {

constexpr int NT = kThreads;
constexpr int NWARP = NT / 32;

template <typename T>
__device__ __forceinline__ T absval(T v) { return v < T(0) ? -v : v; }

// Unblocked LU with partial pivoting of the shared-memory panel P
// (column-major, ld ldp, mp rows, nbk columns).  piv[j] is the panel row
// swapped with row j.  The first exact zero pivot sets *info (1-based,
// offset k0) and leaves that column unscaled, like LAPACK getrf.
template <typename T>
__device__ void panel_factor(T *__restrict__ P, int ldp, int mp, int nbk, int *piv, int k0,
                             int *info, T *redv, int *redi) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = 0; j < nbk; ++j) {
        T best = T(-1);
        int bi = j;
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
        if (lane == 0) { redv[warp] = best; redi[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            best = lane < NWARP ? redv[lane] : T(-1);
            bi = lane < NWARP ? redi[lane] : 0x7fffffff;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) piv[j] = bi;
        }
        __syncthreads();
        const int pr = piv[j];
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
            if (tid == 0 && *info == 0) *info = k0 + j + 1;
        } else {
            const T inv = T(1) / pv;
            for (int i = j + 1 + tid; i < mp; i += NT) {
                const T l = P[j * ldp + i] * inv;
                P[j * ldp + i] = l;
                for (int c = j + 1; c < nbk; ++c) P[c * ldp + i] -= l * P[c * ldp + j];
            }
        }
        __syncthreads();
    }
}

// Mg[r, c0 + c] -= sum_kk A[kk*lda + r - arow0] * B[kk*ldb + c]
// for r in [r0, r1), c in [0, cw); register tiles of TM x TN per thread.
template <typename T, int TM, int TN>
__device__ void gemm_update(T *__restrict__ Mg, int LDC, int r0, int r1, int c0, int cw,
                            const T *__restrict__ A, int lda, int arow0,
                            const T *__restrict__ B, int ldb, int K) {
    constexpr int TX = 16, TY = NT / TX;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    for (int rb = r0; rb < r1; rb += TY * TM) {
        for (int cb = 0; cb < cw; cb += TX * TN) {
            T acc[TM][TN];
#pragma unroll
            for (int u = 0; u < TM; ++u)
#pragma unroll
                for (int v = 0; v < TN; ++v) acc[u][v] = T(0);
            int ra[TM];
#pragma unroll
            for (int u = 0; u < TM; ++u) {
                const int r = rb + ty + u * TY;
                ra[u] = (r < r1 ? r : r0) - arow0;
            }
            for (int kk = 0; kk < K; ++kk) {
                T a[TM], b[TN];
#pragma unroll
                for (int u = 0; u < TM; ++u) a[u] = A[kk * lda + ra[u]];
#pragma unroll
                for (int v = 0; v < TN; ++v) {
                    const int c = cb + tx + v * TX;
                    b[v] = c < cw ? B[kk * ldb + c] : T(0);
                }
#pragma unroll
                for (int u = 0; u < TM; ++u)
#pragma unroll
                    for (int v = 0; v < TN; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
            }
#pragma unroll
            for (int u = 0; u < TM; ++u) {
                const int r = rb + ty + u * TY;
                if (r >= r1) continue;
                T *row = Mg + (long long)r * LDC + c0;
#pragma unroll
                for (int v = 0; v < TN; ++v) {
                    const int c = cb + tx + v * TX;
                    if (c < cw) row[c] -= acc[u][v];
                }
            }
        }
    }
}

template <typename T> struct Tile { static constexpr int M = 4, N = 4; };

struct Smem {
    void *Ps, *Us;
    int *piv, *redi, *misc;
    void *redv;
};

__device__ Smem carve(unsigned char *base, const LuBlocking &P, size_t tsize) {
    Smem s;
    s.Ps = base;
    s.Us = base + (size_t)P.nb_panel * P.ldp * tsize;
    unsigned char *ip = base + (size_t)P.nb_panel * (P.ldp + P.ch) * tsize;
    ip = (unsigned char *)(((uintptr_t)ip + 15) & ~(uintptr_t)15);
    s.redv = ip;                 // NWARP entries of up to 8 bytes
    s.piv = (int *)(ip + 64);    // nb_panel entries (<= 64)
    s.redi = s.piv + 64;         // NWARP entries
    s.misc = s.redi + 16;        // scratch scalars
    return s;
}

// Blocked elimination on the augmented matrix M = [A | RHS] (row-major,
// n rows, C columns).  factor = true: factor A in place (L strictly below
// the diagonal, U on and above; pivots to piv_g if non-null) while
// eliminating every column to the right.  factor = false: replay the stored
// factors and pivots on the right-hand columns [n, C) only.  Then solve
// U X = Y in place for X in columns [n, C).
template <typename T>
__device__ void lu_solve(T *__restrict__ M, int LDC, int n, int C, bool factor, int *piv_g,
                         const LuBlocking &P, const Smem &sm) {
    T *Ps = (T *)sm.Ps;
    T *Us = (T *)sm.Us;
    int *piv = sm.piv;
    const int NB = P.nb_panel, ldp = P.ldp, CH = P.ch;
    const int tid = threadIdx.x;
    constexpr int TM = Tile<T>::M, TN = Tile<T>::N;

    for (int k0 = 0; k0 < n; k0 += NB) {
        const int nbk = min(NB, n - k0), mp = n - k0;
        for (int e = tid; e < mp * nbk; e += NT) {
            const int rr = e / nbk, cc = e % nbk;
            Ps[cc * ldp + rr] = M[(long long)(k0 + rr) * LDC + k0 + cc];
        }
        if (!factor) {
            for (int j = tid; j < nbk; j += NT) piv[j] = piv_g[k0 + j] - k0;
        }
        __syncthreads();
        if (factor) {
            panel_factor<T>(Ps, ldp, mp, nbk, piv, k0, &sm.misc[1], (T *)sm.redv, sm.redi);
            for (int e = tid; e < mp * nbk; e += NT) {
                const int rr = e / nbk, cc = e % nbk;
                M[(long long)(k0 + rr) * LDC + k0 + cc] = Ps[cc * ldp + rr];
            }
            if (piv_g)
                for (int j = tid; j < nbk; j += NT) piv_g[k0 + j] = k0 + piv[j];
        }
        const int cstart = factor ? k0 + nbk : n;
        for (int c0 = cstart; c0 < C; c0 += CH) {
            const int cw = min(CH, C - c0);
            for (int cc = tid; cc < cw; cc += NT) {
                T *col = M + c0 + cc;
                for (int j = 0; j < nbk; ++j) {
                    const int pr = k0 + piv[j];
                    if (pr != k0 + j) {
                        const T a = col[(long long)(k0 + j) * LDC];
                        col[(long long)(k0 + j) * LDC] = col[(long long)pr * LDC];
                        col[(long long)pr * LDC] = a;
                    }
                }
                for (int j = 0; j < nbk; ++j) {
                    T v = col[(long long)(k0 + j) * LDC];
                    for (int i2 = 0; i2 < j; ++i2) v -= Ps[i2 * ldp + j] * Us[i2 * CH + cc];
                    Us[j * CH + cc] = v;
                    col[(long long)(k0 + j) * LDC] = v;
                }
            }
            __syncthreads();
            gemm_update<T, TM, TN>(M, LDC, k0 + nbk, n, c0, cw, Ps, ldp, k0, Us, CH, nbk);
            __syncthreads();
        }
    }

    // Backward substitution, block rows from the bottom.
    for (int kb0 = ((n - 1) / NB) * NB; kb0 >= 0; kb0 -= NB) {
        const int nbk = min(NB, n - kb0), rows = kb0 + nbk;
        for (int e = tid; e < rows * nbk; e += NT) {
            const int rr = e / nbk, cc = e % nbk;
            Ps[cc * ldp + rr] = M[(long long)rr * LDC + kb0 + cc];
        }
        __syncthreads();
        for (int c0 = n; c0 < C; c0 += CH) {
            const int cw = min(CH, C - c0);
            for (int cc = tid; cc < cw; cc += NT) {
                T *col = M + c0 + cc;
                for (int j = nbk - 1; j >= 0; --j) {
                    T v = col[(long long)(kb0 + j) * LDC];
                    for (int i2 = j + 1; i2 < nbk; ++i2) v -= Ps[i2 * ldp + kb0 + j] * Us[i2 * CH + cc];
                    v = v / Ps[j * ldp + kb0 + j];
                    Us[j * CH + cc] = v;
                    col[(long long)(kb0 + j) * LDC] = v;
                }
            }
            __syncthreads();
            gemm_update<T, TM, TN>(M, LDC, 0, kb0, c0, cw, Ps, ldp, 0, Us, CH, nbk);
            __syncthreads();
        }
    }
}



}  // namespace lu
}  // namespace hps
