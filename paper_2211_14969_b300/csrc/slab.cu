// SlabLU (Section 2 of arXiv 2211.14969, the slab block form of Eq. (dell1)):
// the reduced system's interface unknowns between slabs of s leaf columns.
//
// Each slab's interior is eliminated by the merge levels inside the slab
// (hps_api.cu), which leaves the slab's DtN map and flux [T | h] on its
// boundary [W (n), E (n), S (sq), N (sq)], n = ny q.  Flux continuity on
// interface k (between slabs k and k+1, k = 0..S-2) reads
//   D_k u_k + L_k u_{k-1} + U_k u_{k+1} = b_k,
//   D_k = T^k_EE + T^{k+1}_WW,  L_k = T^k_EW,  U_k = T^{k+1}_WE,
//   b_k = -(h^k_E + h^{k+1}_W) - (Dirichlet terms of the outer boundary),
// block tridiagonal.  Block LU with explicit operators, so that solving for
// new Dirichlet data needs only matrix-vector products:
//   Delta_k = D_k + L_k S_{k-1},  [S_k | G_k | v_k] = Delta_k^{-1} [-U_k | I | b^h_k - L_k v_{k-1}],
// and then u_k = v_k + v^g_k + S_k u_{k+1} with v^g_k = G_k (b^g_k - L_k v^g_{k-1}).
// The kernels here form the augmented systems [Delta_k | 0 | -U_k | I | y_k]
// (solved in place by the many-CTA dense solve of merge_split.cu), apply the
// stored operators, and gather each slab's boundary values for the
// downward pass inside the slabs.
#include <cuda_runtime.h>

#include <algorithm>

#include "hps_internal.cuh"
#include "merge.cuh"

namespace hps {
namespace {

constexpr int NT = 256;

// [Delta_k | y_k] = [D_k | b^h_k] + L_k [S_{k-1} | -v_{k-1}]   (n x (n + m))
// written to aug_k columns [0, n) and [c3 + 2n, c3 + 2n + m).  Tiles of
// 64 x 64 outputs, 4 x 4 per thread, K = n staged through shared memory;
// prev == nullptr (the first interface) skips the product.
__global__ void __launch_bounds__(NT) slab_assemble(SlabStepDev S) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int n = S.n, m = S.m, ldt = S.ldt, lda = S.lda, c3 = S.c3;
    const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
    if (S.prev) {
        const double *Lk = S.left + (long long)n * ldt;   // slab k, E rows, W columns
        for (int k0 = 0; k0 < n; k0 += BK) {
            for (int e = threadIdx.x; e < BK * BM; e += NT) {
                const int kk = e / BM, rr = e % BM, i = r0 + rr, j = k0 + kk;
                As[kk][rr] = (i < n && j < n) ? Lk[(long long)i * ldt + j] : 0.0;
            }
            for (int e = threadIdx.x; e < BK * BN; e += NT) {
                const int kk = e / BN, cc = e % BN, j = k0 + kk, c = c0 + cc;
                double v = 0.0;
                if (j < n && c < n) v = S.prev[(long long)j * lda + c3 + c];
                else if (j < n && c < n + m) v = -S.prev[(long long)j * lda + c3 + 2 * n + (c - n)];
                Bs[kk][cc] = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                double a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) a[u] = As[kk][ty + 16 * u];
#pragma unroll
                for (int v = 0; v < 4; ++v) b[v] = Bs[kk][tx + 16 * v];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
            }
            __syncthreads();
        }
    }
    const double *TkE = S.left + (long long)n * ldt;      // slab k, E rows
    const double *Tk1W = S.right;                          // slab k+1, W rows
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = r0 + ty + 16 * u;
        if (i >= n) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int c = c0 + tx + 16 * v;
            if (c >= n + m) continue;
            if (c < n) {
                S.aug[(long long)i * lda + c] = TkE[(long long)i * ldt + n + c] + Tk1W[(long long)i * ldt + c] + acc[u][v];
            } else {
                const int cc = c - n;
                const double bh = -(TkE[(long long)i * ldt + S.np + cc] + Tk1W[(long long)i * ldt + S.np + cc]);
                S.aug[(long long)i * lda + c3 + 2 * n + cc] = bh + acc[u][v];
            }
        }
    }
}

// aug_k columns [n, c3) zero, [c3, c3 + n) -U_k (zero for the last
// interface, whose right neighbour is the outer boundary), [c3 + n, c3 + 2n) I.
__global__ void slab_fill(SlabStepDev S) {
    const int n = S.n, lda = S.lda, c3 = S.c3;
    const long long tot = (long long)n * (c3 - n + 2 * n);
    for (long long e = blockIdx.x * (long long)NT + threadIdx.x; e < tot; e += (long long)gridDim.x * NT) {
        const int i = (int)(e / (c3 + n)), c = n + (int)(e % (c3 + n));
        double v = 0.0;
        if (c >= c3 && c < c3 + n) {
            if (S.last == 0) v = -S.right[(long long)i * S.ldt + n + (c - c3)];   // slab k+1: W rows, E columns
        } else if (c >= c3 + n) {
            v = (c - c3 - n) == i ? 1.0 : 0.0;
        }
        S.aug[(long long)i * lda + c] = v;
    }
}

// y[i][c] = beta y[i][c] + alpha sum_j A[i][j] x[j][c] (+ add[i][c]): a warp
// per row, lanes along j, up to 4 right-hand columns per pass.
__global__ void __launch_bounds__(NT) gemv_rows(const double *__restrict__ A, long long lda, int rows, int cols,
                                                const double *__restrict__ x, int ldx, double *y, int ldy, int m,
                                                double alpha, double beta, const double *add, int ldadd) {
    const int i = blockIdx.x * (NT / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (i >= rows) return;
    const double *a = A + (long long)i * lda;
    for (int c0 = 0; c0 < m; c0 += 4) {
        const int nc = m - c0 < 4 ? m - c0 : 4;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int j = lane; j < cols; j += 32) {
            const double aj = a[j];
            const double *xr = x + (long long)j * ldx + c0;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c < nc) acc[c] = fma(aj, xr[c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o);
        if (lane == 0)
            for (int c = 0; c < nc; ++c) {
                double v = alpha * acc[c];
                if (beta != 0.0) v += beta * y[(long long)i * ldy + c0 + c];
                if (add) v += add[(long long)i * ldadd + c0 + c];
                y[(long long)i * ldy + c0 + c] = v;
            }
    }
}

// Boundary values of every slab [W (n), E (n), S (sq), N (sq)] x m from the
// interface values u (S-1 blocks of n x m) and the outer Dirichlet data g in
// the grid's root order [W (n), E (n), S (nx q), N (nx q)].
__global__ void slab_bounds(int nslab, int n, int sq, int nxq, int m, const double *__restrict__ u,
                            const double *__restrict__ g, double *__restrict__ ub) {
    const int j = blockIdx.y, np = 2 * n + 2 * sq;
    for (int e = blockIdx.x * NT + threadIdx.x; e < np * m; e += gridDim.x * NT) {
        const int r = e / m, c = e % m;
        double v;
        if (r < n) v = j == 0 ? g[(long long)r * m + c] : u[((long long)(j - 1) * n + r) * m + c];
        else if (r < 2 * n) v = j == nslab - 1 ? g[(long long)r * m + c] : u[((long long)j * n + (r - n)) * m + c];
        else if (r < 2 * n + sq) v = g[(long long)(2 * n + j * sq + (r - 2 * n)) * m + c];
        else v = g[(long long)(2 * n + nxq + j * sq + (r - 2 * n - sq)) * m + c];
        ub[(long long)j * np * m + e] = v;
    }
}

}  // namespace

cudaError_t launch_slab_assemble(const SlabStepDev &S, cudaStream_t s) {
    dim3 grid((S.n + S.m + 63) / 64, (S.n + 63) / 64);
    slab_assemble<<<grid, NT, 0, s>>>(S);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long tot = (long long)S.n * (S.c3 + S.n);
    slab_fill<<<(int)std::min<long long>((tot + NT - 1) / NT, 2048), NT, 0, s>>>(S);
    return cudaGetLastError();
}

cudaError_t launch_gemv(const double *A, long long lda, int rows, int cols, const double *x, int ldx, double *y,
                        int ldy, int m, double alpha, double beta, const double *add, int ldadd, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    gemv_rows<<<(rows + NT / 32 - 1) / (NT / 32), NT, 0, s>>>(A, lda, rows, cols, x, ldx, y, ldy, m, alpha, beta, add,
                                                             ldadd);
    return cudaGetLastError();
}

cudaError_t launch_slab_bounds(int nslab, int n, int sq, int nxq, int m, const double *u, const double *g, double *ub,
                               cudaStream_t s) {
    const int np = 2 * n + 2 * sq;
    slab_bounds<<<dim3((np * m + NT - 1) / NT, nslab), NT, 0, s>>>(nslab, n, sq, nxq, m, u, g, ub);
    return cudaGetLastError();
}

}  // namespace hps
