// Dense solves of the upper merge levels spread over many CTAs.
//
// A merge solves Z X = B with Z = Ta33 + Tb33 (n3 x n3) and
// B = -[Ta31 Tb32 | ha3 + hb3]; the HPS merge of two boxes (Section 2 of
// arXiv 2211.14969 takes it from its references).  Near the root of a
// uniform tree there are few merges and each is large (a 64 x 64 grid of
// p = 20 leaves ends with one merge of n3 = 1152 and 4609 right-hand
// columns), so one CTA per merge would leave all but a handful of SMs
// idle.  Here every level with few merges runs a right-looking blocked LU
// with partial pivoting on the augmented row-major matrix
// [Z | 0 | B] -> [U | 0 | X], one launch per step, with the work of each
// step spread over column blocks and 64 x 64 output tiles:
//
//   for each panel of NB columns at k:
//     panel:      factor rows k.. of columns k..k+NB-1 (one CTA per merge,
//                 panel in shared memory, block-wide argmax per column);
//     swap_lower: apply the panel's interchanges to the columns right of the
//                 panel and solve the unit-lower L11 for the NB rows at k
//                 (one thread per column);
//     gemm:       A22 -= L21 U12, the next panel's columns first (64 x 16
//                 tiles) and the rest (64 x 64 tiles) on a second stream,
//                 where it overlaps the next panel's factorization;
//   then for each block row kb from the bottom:
//     upper:      X1 = U11^{-1} Y1 on the NB rows at kb (thread per column);
//     gemm:       Y0 -= U01 X1 on the rows above.
//
// The multipliers of L are not applied to earlier columns: the right-hand
// side is eliminated together with Z, so L is never needed again and the
// columns left of a panel keep its multipliers in their unswapped rows.
//
// With oz_solve (large interfaces, tensor path on) the steps above touch
// only Z's columns; the right-hand side is eliminated per block of
// kSplitKB rows instead: the block's interchanges in order (split_swap_cols,
// which also applies each panel's interchanges to the block's earlier L
// columns), its unit-lower solve in one kernel (split_block_trsm), and one
// FP64-accurate tensor-core update of all rows below (ozaki.cu); the back
// substitution likewise per block from the bottom, updating the rows above.
// Panels are 16 columns wide, 8 where 16 do not fit the panel kernel's
// shared memory (interfaces of 1601 to 3200 nodes).
// info[s] receives the first step with an exactly zero pivot (1-based),
// as LAPACK's getrf does; the elimination then continues without scaling.
#include <cuda_runtime.h>

#include "merge.cuh"

namespace hps {
namespace {

constexpr int PNT = 256;   // threads of the panel kernel
constexpr int CNT = 128;   // threads (columns) of the triangular kernels
constexpr int GT = 64;     // gemm output tile (GT x GT), 256 threads, 4 x 4 each

// Panel factorization.  P (column-major, ld = odd >= rows) holds rows
// k..n3-1 of columns k..k+nbk-1.
template <int NB>
__global__ void __launch_bounds__(PNT) split_panel(double *__restrict__ aug, long long stride, int n3, int lda,
                                                   int k, int nbk, int *__restrict__ ipiv, int *__restrict__ info) {
    extern __shared__ double P[];
    __shared__ double wv[PNT / 32];
    __shared__ int wi[PNT / 32];
    __shared__ int pivs;
    const int s = blockIdx.x;
    double *A = aug + (long long)s * stride;
    const int rows = n3 - k;
    const int ld = rows | 1;
    for (int e = threadIdx.x; e < rows * NB; e += PNT) {
        const int r = e / NB, c = e % NB;
        P[c * ld + r] = c < nbk ? A[(long long)(k + r) * lda + k + c] : 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < nbk; ++j) {
        // argmax |P[j.., j]|, ties to the smallest row
        double best = -1.0;
        int bi = rows;
        for (int r = j + threadIdx.x; r < rows; r += PNT) {
            const double v = fabs(P[j * ld + r]);
            if (v > best) { best = v; bi = r; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { wv[warp] = best; wi[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = wv[0];
            int i = wi[0];
            for (int w = 1; w < PNT / 32; ++w)
                if (wv[w] > b || (wv[w] == b && wi[w] < i)) { b = wv[w]; i = wi[w]; }
            if (!(b > 0.0)) {
                i = j;  // exact zero column: no interchange, no scaling
                if (info[s] == 0) info[s] = k + j + 1;
            }
            pivs = i;
            ipiv[(long long)s * n3 + k + j] = k + i;
        }
        __syncthreads();
        const int pr = pivs;
        if (pr != j) {
            for (int c = threadIdx.x; c < nbk; c += PNT) {
                const double t = P[c * ld + j];
                P[c * ld + j] = P[c * ld + pr];
                P[c * ld + pr] = t;
            }
            __syncthreads();
        }
        const double d = P[j * ld + j];
        if (d != 0.0) {
            const double rd = 1.0 / d;
            for (int r = j + 1 + threadIdx.x; r < rows; r += PNT) {
                const double l = P[j * ld + r] * rd;
                P[j * ld + r] = l;
                for (int c = j + 1; c < nbk; ++c) P[c * ld + r] = fma(-l, P[c * ld + j], P[c * ld + r]);
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < rows * nbk; e += PNT) {
        const int r = e / nbk, c = e % nbk;
        A[(long long)(k + r) * lda + k + c] = P[c * ld + r];
    }
}

// Interchanges and the unit-lower solve for the columns right of the panel.
template <int NB>
__global__ void __launch_bounds__(CNT) split_swap_lower(double *__restrict__ aug, long long stride, int n3, int lda,
                                                        int k, int nbk, int c0, int C, const int *__restrict__ ipiv,
                                                        int swap) {
    __shared__ double L[NB][NB];
    __shared__ int pv[NB];
    const int s = blockIdx.y;
    double *A = aug + (long long)s * stride;
    for (int e = threadIdx.x; e < NB * NB; e += CNT) {
        const int i = e / NB, j = e % NB;
        L[i][j] = (i < nbk && j < nbk) ? A[(long long)(k + i) * lda + k + j] : 0.0;
    }
    if (threadIdx.x < NB) pv[threadIdx.x] = threadIdx.x < nbk ? ipiv[(long long)s * n3 + k + threadIdx.x] : 0;
    __syncthreads();
    const int col = c0 + blockIdx.x * CNT + threadIdx.x;
    if (col >= C) return;
    double x[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (swap && j < nbk) {
            const int r = pv[j];
            double *a = A + (long long)(k + j) * lda + col;
            if (r != k + j) {
                double *b = A + (long long)r * lda + col;
                const double t = *a;
                *a = *b;
                *b = t;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (j < nbk) {
            double v = A[(long long)(k + j) * lda + col];
#pragma unroll
            for (int i = 0; i < j; ++i) v = fma(-L[j][i], x[i], v);
            x[j] = v;
        } else {
            x[j] = 0.0;
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (j < nbk) A[(long long)(k + j) * lda + col] = x[j];
}

// The interchanges of pivot steps k..k+np-1, in order, for the columns
// [c0, c1): a block's L columns left of its panel, or the right-hand side
// once per elimination block.
__global__ void __launch_bounds__(CNT) split_swap_cols(double *__restrict__ aug, long long stride, int n3, int lda,
                                                       int k, int np, int c0, int c1, const int *__restrict__ ipiv) {
    const int s = blockIdx.y;
    const int col = c0 + blockIdx.x * CNT + threadIdx.x;
    if (col >= c1) return;
    double *A = aug + (long long)s * stride + col;
    const int *pv = ipiv + (long long)s * n3 + k;
    for (int j = 0; j < np; ++j) {
        const int r = pv[j];
        if (r != k + j) {
            const double t = A[(long long)(k + j) * lda];
            A[(long long)(k + j) * lda] = A[(long long)r * lda];
            A[(long long)r * lda] = t;
        }
    }
}

// The triangular solve of one elimination block for the right-hand side:
// rows [b0, b0 + nb) of the columns [c0, C), nb <= kSplitKB, in place;
// UPPER: X = U^{-1} Y with the block's upper triangle, else Y = L^{-1} Y
// with its unit-lower triangle.  A CTA holds the triangle and a slab of
// TW columns in shared memory; thread t updates column t % TW and the rows
// congruent to t / TW modulo 256 / TW, one pivot row after the other.
constexpr int TW = 32;
template <bool UPPER>
__global__ void __launch_bounds__(256, 1) split_block_trsm(double *__restrict__ aug, long long stride, int lda, int b0,
                                                           int nb, int c0, int C) {
    extern __shared__ double sm[];
    const int ldt = nb | 1;
    double *Tr = sm;                            // [nb][ldt]
    double *Y = sm + (size_t)nb * ldt;          // [nb][TW]
    double *rd = Y + (size_t)nb * TW;           // [nb] reciprocals of U's diagonal
    const int s = blockIdx.y, cb = c0 + blockIdx.x * TW;
    const double *A = aug + (long long)s * stride;
    for (int e = threadIdx.x; e < nb * nb; e += 256) {
        const int i = e / nb, j = e % nb;
        Tr[i * ldt + j] = A[(long long)(b0 + i) * lda + b0 + j];
    }
    for (int e = threadIdx.x; e < nb * TW; e += 256) {
        const int i = e / TW, c = e % TW;
        Y[e] = cb + c < C ? A[(long long)(b0 + i) * lda + cb + c] : 0.0;
    }
    if (UPPER)
        for (int j = threadIdx.x; j < nb; j += 256) rd[j] = 1.0 / A[(long long)(b0 + j) * lda + b0 + j];
    __syncthreads();
    const int c = threadIdx.x % TW, r0 = threadIdx.x / TW;
    constexpr int RS = 256 / TW;   // rows per thread step; row i belongs to the threads with r0 = i % RS
    if (!UPPER) {
        for (int j = 0; j < nb - 1; ++j) {
            const double x = Y[j * TW + c];
            for (int i = j + 1 + ((r0 - (j + 1)) % RS + RS) % RS; i < nb; i += RS)
                Y[i * TW + c] = fma(-Tr[i * ldt + j], x, Y[i * TW + c]);
            __syncthreads();
        }
    } else {
        // the row's owner scales it by the diagonal's reciprocal (one division
        // per row and CTA: the FP64 pipe is the bound here), then the rows
        // above are updated
        for (int j = nb - 1; j >= 0; --j) {
            if (r0 == j % RS) Y[j * TW + c] *= rd[j];
            __syncthreads();
            const double x = Y[j * TW + c];
            for (int i = r0; i < j; i += RS) Y[i * TW + c] = fma(-Tr[i * ldt + j], x, Y[i * TW + c]);
        }
        __syncthreads();
    }
    double *W = aug + (long long)s * stride;
    for (int e = threadIdx.x; e < nb * TW; e += 256) {
        const int i = e / TW, cc = e % TW;
        if (cb + cc < C) W[(long long)(b0 + i) * lda + cb + cc] = Y[e];
    }
}

// X1 = U11^{-1} Y1 for the right-hand columns of block row kb.
template <int NB>
__global__ void __launch_bounds__(CNT) split_upper(double *__restrict__ aug, long long stride, int lda, int kb, int nbk,
                                                   int c0, int C) {
    __shared__ double U[NB][NB];
    const int s = blockIdx.y;
    double *A = aug + (long long)s * stride;
    for (int e = threadIdx.x; e < NB * NB; e += CNT) {
        const int i = e / NB, j = e % NB;
        U[i][j] = (i < nbk && j < nbk) ? A[(long long)(kb + i) * lda + kb + j] : 1.0;
    }
    __syncthreads();
    const int col = c0 + blockIdx.x * CNT + threadIdx.x;
    if (col >= C) return;
    double x[NB];
#pragma unroll
    for (int j = NB - 1; j >= 0; --j) {
        if (j < nbk) {
            double v = A[(long long)(kb + j) * lda + col];
#pragma unroll
            for (int i = j + 1; i < NB; ++i)
                if (i < nbk) v = fma(-U[j][i], x[i], v);
            x[j] = v / U[j][j];
        } else {
            x[j] = 0.0;
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (j < nbk) A[(long long)(kb + j) * lda + col] = x[j];
}

// C[r0 + i][c0 + j] -= sum_t A[r0 + i][ka + t] * A[kb + t][c0 + j], t < K <= KM,
// over GT x GT tiles of the nr x nc block (all inside one merge's matrix).
template <int KM>
__global__ void __launch_bounds__(256) split_gemm(double *__restrict__ aug, long long stride, int lda, int r0, int nr,
                                                  int c0, int nc, int ka, int kb, int K) {
    __shared__ double As[KM][GT + 1];
    __shared__ double Bs[KM][GT];
    const int s = blockIdx.z;
    double *A = aug + (long long)s * stride;
    const int tr = blockIdx.y * GT, tc = blockIdx.x * GT;
    for (int e = threadIdx.x; e < GT * KM; e += 256) {
        const int i = e / KM, t = e % KM;
        As[t][i] = (tr + i < nr && t < K) ? A[(long long)(r0 + tr + i) * lda + ka + t] : 0.0;
    }
    for (int e = threadIdx.x; e < KM * GT; e += 256) {
        const int t = e / GT, j = e % GT;
        Bs[t][j] = (t < K && tc + j < nc) ? A[(long long)(kb + t) * lda + c0 + tc + j] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // outputs (ty + 16u, tx + 16v)
    double acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
#pragma unroll
    for (int t = 0; t < KM; ++t) {
        double a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = As[t][ty + 16 * u];
#pragma unroll
        for (int v = 0; v < 4; ++v) b[v] = Bs[t][tx + 16 * v];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = tr + ty + 16 * u;
        if (i >= nr) continue;
        double *row = A + (long long)(r0 + i) * lda + c0 + tc;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int j = tx + 16 * v;
            if (tc + j < nc) row[j] -= acc[u][v];
        }
    }
}

// The same update for a block at most 16 columns wide (the next panel's
// columns in the look-ahead): 64 x 16 tiles, 4 outputs per thread.
template <int KM>
__global__ void __launch_bounds__(256) split_gemm_n16(double *__restrict__ aug, long long stride, int lda, int r0,
                                                      int nr, int c0, int nc, int ka, int kb, int K) {
    __shared__ double As[KM][GT + 1];
    __shared__ double Bs[KM][16];
    const int s = blockIdx.z;
    double *A = aug + (long long)s * stride;
    const int tr = blockIdx.y * GT;
    for (int e = threadIdx.x; e < GT * KM; e += 256) {
        const int i = e / KM, t = e % KM;
        As[t][i] = (tr + i < nr && t < K) ? A[(long long)(r0 + tr + i) * lda + ka + t] : 0.0;
    }
    for (int e = threadIdx.x; e < KM * 16; e += 256) {
        const int t = e / 16, j = e % 16;
        Bs[t][j] = (t < K && j < nc) ? A[(long long)(kb + t) * lda + c0 + j] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // outputs (ty + 16u, tx)
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int t = 0; t < KM; ++t) {
        const double b = Bs[t][tx];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fma(As[t][ty + 16 * u], b, acc[u]);
    }
    if (tx >= nc) return;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = tr + ty + 16 * u;
        if (i < nr) A[(long long)(r0 + i) * lda + c0 + tx] -= acc[u];
    }
}

}  // namespace

constexpr int kSplitKB = 128;   // elimination block of the right-hand side with oz_solve (a multiple of the panel width)

// panel width: 16 columns while a panel of the whole height fits the
// panel kernel's shared memory, else 8 (interfaces of up to 3200 nodes)
static bool panel_fits(int n3, int nb) { return (size_t)((n3 | 1) * nb) * sizeof(double) <= 200 * 1024; }
static int split_nb(int n3) { return panel_fits(n3, 16) ? 16 : 8; }
bool split_solve_fits(int n3) { return panel_fits(n3, 8); }

bool split_solve_blocked(int n3, int nrhs) { return n3 >= 2 * kSplitKB && n3 <= 8192 && nrhs >= kSplitKB; }

size_t split_solve_scratch(int nm, int n3, int nrhs) { return ozaki_scratch_bytes(nm, n3, kSplitKB, nrhs); }

// the kernels launch_split_solve issues (an Ozaki job is four)
int split_solve_launches(int n3, int nrhs, bool blocked, bool aux) {
    const int NB = split_nb(n3);
    const int CZ = blocked ? n3 : n3 + nrhs;   // columns past the panel the LU steps touch, counted from 0
    int n = 0, kb0 = 0;
    for (int k = 0; k < n3; k += NB) {
        const int nbk = n3 - k < NB ? n3 - k : NB;
        const int cr = CZ - (k + nbk), nr = n3 - (k + nbk);
        n += 1 + (cr > 0) + (blocked && k > kb0);
        if (nr > 0 && cr > 0) n += (aux && cr > (nr < NB ? nr : NB)) ? 2 : 1;
        const int kb1 = k + nbk;
        if (blocked && (kb1 - kb0 == kSplitKB || kb1 == n3)) {
            n += 2;   // interchanges, block solve
            if (kb1 < n3) n += 4;
            kb0 = kb1;
        }
    }
    if (!blocked) return n + 2 * ((n3 + NB - 1) / NB) - 1;
    for (int b0 = ((n3 - 1) / kSplitKB) * kSplitKB; b0 >= 0; b0 -= kSplitKB) {
        n += 1 + (b0 > 0 ? 4 : 0);
    }
    return n;
}

template <int NB>
static cudaError_t split_solve_nb(const MergeLevelDev &L, int *ipiv, cudaStream_t st, const SplitAux *aux) {
    const int n3 = L.n3, lda = L.lda, nm = L.nm;
    const int C = L.c3 + L.np + L.m;
    const long long stride = (long long)n3 * lda;
    if (ipiv == nullptr || !panel_fits(n3, NB)) return cudaErrorInvalidValue;
    const size_t psmem = (size_t)((n3 | 1) * NB) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(split_panel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(L.info, 0, (size_t)nm * sizeof(int), st)) != cudaSuccess) return e;
    auto trsm_smem = [](int nb) { return (size_t)nb * ((nb | 1) + TW + 1) * sizeof(double); };
    if (L.oz_solve) {
        const int mx = (int)trsm_smem(kSplitKB);
        if ((e = cudaFuncSetAttribute(split_block_trsm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) !=
                cudaSuccess ||
            (e = cudaFuncSetAttribute(split_block_trsm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)) !=
                cudaSuccess)
            return e;
    }
    auto gemm = [&](cudaStream_t s, int r0, int nr, int c0, int nc, int ka, int kb, int K) {
        split_gemm<NB><<<dim3((nc + GT - 1) / GT, (nr + GT - 1) / GT, nm), 256, 0, s>>>(L.aug, stride, lda, r0, nr, c0,
                                                                                        nc, ka, kb, K);
    };
    const int nrhs = C - L.c3;
    // With oz_solve the LU steps eliminate only Z's columns; the right-hand
    // side is eliminated per block of kSplitKB rows (interchanges, the
    // block's unit-lower solve, then one tensor-core update of every row
    // below it), as in a blocked LU solve.
    const bool blocked = L.oz_solve != 0;
    const int CZ = blocked ? n3 : C;   // last column the LU steps touch
    auto rhs_update = [&](int r0, int M, int k0, int K) -> cudaError_t {
        OzJob J{};
        J.nm = nm;
        J.M = M;
        J.K = K;
        J.N = nrhs;
        J.a = L.aug + (long long)r0 * lda + k0;
        J.sa = stride;
        J.lda = lda;
        J.b = L.aug + (long long)k0 * lda + L.c3;
        J.sb = stride;
        J.ldb = lda;
        J.c = L.aug + (long long)r0 * lda + L.c3;
        J.sc = stride;
        J.ldc = lda;
        return launch_ozaki(J, L.oz, st);
    };
    // With aux, look-ahead: each step first updates only the next panel's
    // columns, and the rest of its trailing update runs on the side stream
    // while the next panel is factored (the two touch disjoint columns); the
    // next step's interchanges wait for it.
    bool pending = false;
    int kb0 = 0;   // first row of the current elimination block
    for (int k = 0; k < n3; k += NB) {
        const int nbk = n3 - k < NB ? n3 - k : NB;
        const size_t sm = (size_t)(((n3 - k) | 1) * NB) * sizeof(double);
        split_panel<NB><<<nm, PNT, sm, st>>>(L.aug, stride, n3, lda, k, nbk, ipiv, L.info);
        if (pending && (e = cudaStreamWaitEvent(st, aux->b, 0)) != cudaSuccess) return e;
        pending = false;
        const int cr = CZ - (k + nbk);
        if (cr > 0)
            split_swap_lower<NB><<<dim3((cr + CNT - 1) / CNT, nm), CNT, 0, st>>>(L.aug, stride, n3, lda, k, nbk, k + nbk,
                                                                                 CZ, ipiv, 1);
        if (blocked && k > kb0)
            split_swap_cols<<<dim3((k - kb0 + CNT - 1) / CNT, nm), CNT, 0, st>>>(L.aug, stride, n3, lda, k, nbk, kb0, k,
                                                                                 ipiv);
        const int nr = n3 - (k + nbk);
        if (nr > 0 && cr > 0) {
            const int next_w = nr < NB ? nr : NB;
            if (aux && cr > next_w) {
                split_gemm_n16<NB><<<dim3(1, (nr + GT - 1) / GT, nm), 256, 0, st>>>(L.aug, stride, lda, k + nbk, nr,
                                                                                    k + nbk, next_w, k, k, nbk);
                if ((e = cudaEventRecord(aux->a, st)) != cudaSuccess) return e;
                if ((e = cudaStreamWaitEvent(aux->side, aux->a, 0)) != cudaSuccess) return e;
                gemm(aux->side, k + nbk, nr, k + nbk + next_w, cr - next_w, k, k, nbk);
                if ((e = cudaEventRecord(aux->b, aux->side)) != cudaSuccess) return e;
                pending = true;
            } else {
                gemm(st, k + nbk, nr, k + nbk, cr, k, k, nbk);
            }
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int kb1 = k + nbk;
        if (blocked && (kb1 - kb0 == kSplitKB || kb1 == n3)) {
            // the right-hand side of block rows [kb0, kb1): its interchanges in
            // order, the unit-lower solve inside the block, the rows below
            split_swap_cols<<<dim3((nrhs + CNT - 1) / CNT, nm), CNT, 0, st>>>(L.aug, stride, n3, lda, kb0, kb1 - kb0,
                                                                              L.c3, C, ipiv);
            split_block_trsm<false><<<dim3((nrhs + TW - 1) / TW, nm), 256, trsm_smem(kb1 - kb0), st>>>(
                L.aug, stride, lda, kb0, kb1 - kb0, L.c3, C);
            if (kb1 < n3 && (e = rhs_update(kb1, n3 - kb1, kb0, kb1 - kb0)) != cudaSuccess) return e;
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            kb0 = kb1;
        }
    }
    if (pending && (e = cudaStreamWaitEvent(st, aux->b, 0)) != cudaSuccess) return e;
    const int last = ((n3 - 1) / NB) * NB;
    if (!blocked) {
        for (int kb = last; kb >= 0; kb -= NB) {
            const int nbk = n3 - kb < NB ? n3 - kb : NB;
            split_upper<NB><<<dim3((nrhs + CNT - 1) / CNT, nm), CNT, 0, st>>>(L.aug, stride, lda, kb, nbk, L.c3, C);
            if (kb > 0) gemm(st, 0, kb, L.c3, nrhs, kb, kb, nbk);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    // back substitution per block from the bottom: inside the block, then
    // one tensor-core update of every row above it
    for (int b0 = ((n3 - 1) / kSplitKB) * kSplitKB; b0 >= 0; b0 -= kSplitKB) {
        const int b1 = b0 + kSplitKB < n3 ? b0 + kSplitKB : n3;
        split_block_trsm<true><<<dim3((nrhs + TW - 1) / TW, nm), 256, trsm_smem(b1 - b0), st>>>(L.aug, stride, lda, b0,
                                                                                             b1 - b0, L.c3, C);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (b0 > 0 && (e = rhs_update(0, b0, b0, b1 - b0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_split_solve(const MergeLevelDev &L, int *ipiv, cudaStream_t st, const SplitAux *aux) {
    return split_nb(L.n3) == 16 ? split_solve_nb<16>(L, ipiv, st, aux) : split_solve_nb<8>(L, ipiv, st, aux);
}

}  // namespace hps
