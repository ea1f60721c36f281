// Upward merges and the top-down solve over a uniform grid of condensed
// leaves (the HPS merge that Section 2 of arXiv 2211.14969 takes from its
// references, and the leaf recovery of the Section 2 Remark).
//
// Per merge of boxes alpha, beta with shared edge 3 and exterior edges 1, 2:
//   [Z | -[Ta31 Tb32] | -(ha3 + hb3)]  --dense LU solve-->  [LU | S3 | w3]
//   T = diag(Ta11, Tb22) + [Ta13; Tb23] S3,   h = [ha1; hb2] + [Ta13; Tb23] w3
// with every index expressed in the parent's boundary order through per-level
// maps built on the host.  Downward: u3 = S3 u_parent + w3, children's
// boundary values gathered from the parent's values and u3, and finally
// u_i = S u_b + W on every leaf.  Levels with few merges solve Z over many
// CTAs (merge_split.cu) instead of one CTA per merge.
#include <cuda_runtime.h>

#include "hps_internal.cuh"
#include "merge.cuh"

namespace hps {
namespace {

constexpr int NT = 256;

struct ChildView {
    const double *T;  // child's DtN map, row-major, ld
    const double *h;  // child's flux, row-major, ldh
    int ld, ldh;
};

__device__ __forceinline__ ChildView child_view(const MergeLevelDev &L, int child) {
    ChildView v;
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

// Aug[s] = [Z | 0 | -[Ta31 Tb32] (parent column order) | -(ha3 + hb3)].
__global__ void merge_build_aug(MergeLevelDev L) {
    const int s = blockIdx.y;
    const ChildView A = child_view(L, L.ca[s]);
    const ChildView B = child_view(L, L.cb[s]);
    double *aug = L.aug + (long long)s * L.n3 * L.lda;
    const int C = L.c3 + L.np + L.m;
    for (long long e = blockIdx.x * (long long)NT + threadIdx.x; e < (long long)L.n3 * C;
         e += (long long)gridDim.x * NT) {
        const int k = (int)(e / C), c = (int)(e % C);
        const int ra = L.s3a[k], rb = L.s3b[k];
        double v;
        if (c < L.n3) {
            v = A.T[(long long)ra * A.ld + L.s3a[c]] + B.T[(long long)rb * B.ld + L.s3b[c]];
        } else if (c < L.c3) {
            v = 0.0;
        } else if (c < L.c3 + L.np) {
            const int P = c - L.c3;
            const int idx = L.par_idx[P];
            v = L.par_child[P] == 0 ? -A.T[(long long)ra * A.ld + idx] : -B.T[(long long)rb * B.ld + idx];
        } else {
            const int cc = c - L.c3 - L.np;
            v = -(A.h[(long long)ra * A.ldh + cc] + B.h[(long long)rb * B.ldh + cc]);
        }
        aug[(long long)k * L.lda + c] = v;
    }
}

// Parent [T | h] = gather + [Ta13; Tb23] [S3 | w3], tiled over 32 x 32
// output blocks with the K = n3 dimension staged through shared memory.
__global__ void __launch_bounds__(NT) merge_parent(MergeLevelDev L) {
    constexpr int BM = 32, BN = 32, BK = 16;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int s = blockIdx.z;
    const ChildView A = child_view(L, L.ca[s]);
    const ChildView B = child_view(L, L.cb[s]);
    const double *aug = L.aug + (long long)s * L.n3 * L.lda;
    const int ldt = L.np + L.m;
    double *Th = L.Th + (long long)s * L.np * ldt;
    const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 2 x 2 outputs each
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int k0 = 0; k0 < L.n3; k0 += BK) {
        for (int e = threadIdx.x; e < BK * BM; e += NT) {
            const int kk = e / BM, rr = e % BM;
            const int P = r0 + rr, k = k0 + kk;
            double v = 0.0;
            if (P < L.np && k < L.n3) {
                const int idx = L.par_idx[P];
                v = L.par_child[P] == 0 ? A.T[(long long)idx * A.ld + L.s3a[k]]
                                        : B.T[(long long)idx * B.ld + L.s3b[k]];
            }
            As[kk][rr] = v;
        }
        for (int e = threadIdx.x; e < BK * BN; e += NT) {
            const int kk = e / BN, cc = e % BN;
            const int k = k0 + kk, c = c0 + cc;
            Bs[kk][cc] = (k < L.n3 && c < ldt) ? aug[(long long)k * L.lda + L.c3 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const double a0 = As[kk][ty], a1 = As[kk][ty + 16];
            const double b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int P = r0 + ty + 16 * u;
        if (P >= L.np) continue;
        const int chi = L.par_child[P], idx = L.par_idx[P];
        const ChildView &X = chi == 0 ? A : B;
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int c = c0 + tx + 16 * v;
            if (c >= ldt) continue;
            double g;
            if (c < L.np) g = (L.par_child[c] == chi) ? X.T[(long long)idx * X.ld + L.par_idx[c]] : 0.0;
            else g = X.h[(long long)idx * X.ldh + (c - L.np)];
            Th[(long long)P * ldt + c] = g + acc[u][v];
        }
    }
}

// u3 = S3 u_parent + w3: a warp per shared-edge row k, lanes along the
// parent's boundary, four right-hand columns at a time.
__global__ void __launch_bounds__(NT) merge_down_u3(MergeLevelDev L, const double *__restrict__ upar) {
    const int s = blockIdx.y;
    const int k = blockIdx.x * (NT / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (k >= L.n3) return;
    const double *row = L.aug + ((long long)s * L.n3 + k) * L.lda + L.c3;
    const double *up = upar + (long long)s * L.np * L.m;
    double *out = L.u3 + ((long long)s * L.n3 + k) * L.m;
    for (int c0 = 0; c0 < L.m; c0 += 4) {
        const int nc = L.m - c0 < 4 ? L.m - c0 : 4;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int P = lane; P < L.np; P += 32) {
            const double a = row[P];
            const double *u = up + (long long)P * L.m + c0;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c < nc) acc[c] = fma(a, u[c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o);
        }
        if (lane == 0)
            for (int c = 0; c < nc; ++c) out[c0 + c] = acc[c] + row[L.np + c0 + c];
    }
}

// The children's boundary values from the parent's values and u3.
__global__ void __launch_bounds__(NT) merge_down_scatter(MergeLevelDev L, const double *__restrict__ upar,
                                                         double *__restrict__ uchild) {
    const int s = blockIdx.y;
    const double *up = upar + (long long)s * L.np * L.m;
    const double *u3 = L.u3 + (long long)s * L.n3 * L.m;
    const long long per = (long long)L.nbc * L.m;
    for (long long e = blockIdx.x * (long long)NT + threadIdx.x; e < 2 * per; e += (long long)gridDim.x * NT) {
        const int chi = (int)(e / per);
        const int r = (int)(e % per), i = r / L.m, c = r % L.m;
        const int child = chi == 0 ? L.ca[s] : L.cb[s];
        const int sidx = (chi == 0 ? L.srca : L.srcb)[i];
        uchild[(long long)child * per + r] = sidx >= 0 ? up[(long long)sidx * L.m + c] : u3[(-sidx - 1) * L.m + c];
    }
}

// u on every node of every leaf: edges from u_b, interior S u_b + W, corners 0.
__global__ void leaf_recover(int p, int m, const double *__restrict__ S, const double *__restrict__ W,
                             const double *__restrict__ ub, double *__restrict__ u) {
    const int leaf = blockIdx.x;
    const int q = p - 2, n = q * q, nbd = 4 * q;
    const double *Sl = S + (long long)leaf * n * nbd;
    const double *Wl = W ? W + (long long)leaf * n * m : nullptr;
    const double *ul = ub + (long long)leaf * nbd * m;
    double *uo = u + (long long)leaf * p * p * m;
    for (int e = threadIdx.x; e < p * p * m; e += NT) {
        const int node = e / m, c = e % m;
        const int i = node / p, j = node % p;
        const bool ei = (i == 0 || i == p - 1), ej = (j == 0 || j == p - 1);
        double v;
        if (ei && ej) {
            v = 0.0;
        } else if (ei || ej) {
            const int b = (i == 0) ? (j - 1) : (i == p - 1) ? (q + j - 1) : (j == 0) ? (2 * q + i - 1) : (3 * q + i - 1);
            v = ul[(long long)b * m + c];
        } else {
            const int r = (i - 1) * q + (j - 1);
            v = Wl ? Wl[(long long)r * m + c] : 0.0;
            const double *Sr = Sl + (long long)r * nbd;
            for (int b = 0; b < nbd; ++b) v = fma(Sr[b], ul[(long long)b * m + c], v);
        }
        uo[e] = v;
    }
}

}  // namespace

cudaError_t launch_merge_level(const MergeLevelDev &L, bool form_parent, cudaStream_t s, const SplitAux *aux) {
    const int C = L.c3 + L.np + L.m;
    long long work = (long long)L.n3 * C;
    int gx = (int)((work + NT - 1) / NT);
    if (gx > 1024) gx = 1024;
    merge_build_aug<<<dim3(gx, L.nm), NT, 0, s>>>(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (L.ipiv)
        e = launch_split_solve(L, L.ipiv, s, aux);
    else
        e = launch_dense_solve(L.aug, (long long)L.n3 * L.lda, L.n3, L.c3, C, L.lda, L.nm, L.info, s);
    if (e != cudaSuccess) return e;
    if (form_parent) {
        if (L.use_oz) return launch_parent_ozaki(L, L.oz, s);
        const int ldt = L.np + L.m;
        dim3 grid((ldt + 31) / 32, (L.np + 31) / 32, L.nm);
        merge_parent<<<grid, NT, 0, s>>>(L);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_merge_down(const MergeLevelDev &L, const double *upar, double *uchild, cudaStream_t s) {
    merge_down_u3<<<dim3((L.n3 + NT / 32 - 1) / (NT / 32), L.nm), NT, 0, s>>>(L, upar);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long work = 2LL * L.nbc * L.m;
    int gx = (int)((work + NT - 1) / NT);
    if (gx > 64) gx = 64;
    merge_down_scatter<<<dim3(gx, L.nm), NT, 0, s>>>(L, upar, uchild);
    return cudaGetLastError();
}

cudaError_t launch_leaf_recover(int n_leaves, int p, int m, const double *S, const double *W,
                                const double *ub, double *u, cudaStream_t s) {
    leaf_recover<<<n_leaves, NT, 0, s>>>(p, m, S, W, ub, u);
    return cudaGetLastError();
}

}  // namespace hps
