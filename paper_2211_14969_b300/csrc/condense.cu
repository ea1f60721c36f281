// Batched leaf static condensation (Section 2 of arXiv 2211.14969):
// per leaf, assemble the Chebyshev collocation operator, eliminate the
// interior nodes by blocked LU with partial pivoting on the augmented matrix
// [A_ii | -A_ib | f_I], back-substitute for X = [S | W], and form the DtN
// map T = N_b + N_i S and the flux h = N_i W.
//
// One persistent launch: every CTA pops leaves from a global work counter
// (largest leaves first) and condenses each one in its own global-memory
// workspace slot.  The current panel and the U12 column chunk are staged in
// shared memory; the trailing updates are register-tiled.
//
// Working types:
//   HPS_FP64        T = double throughout.
//   HPS_MIXED_FP32  T = float for the LU and both triangular solves, then
//                   FP64 iterative refinement: the residual R = B - A_ii X
//                   is applied matrix-free from the FP64 differentiation
//                   matrices and coefficients, the correction is solved with
//                   the stored FP32 factors, and X is kept in FP64.  S, T, W
//                   and h are written from the FP64 iterate.
#include <cuda_runtime.h>

#include "hps_internal.cuh"
#include "dense_lu.cuh"

namespace hps {
namespace {

using namespace lu;

// Node (k, l) of the n_b-th edge node: edges [W, E, S, N], each by
// increasing coordinate, corners excluded.
__device__ __forceinline__ void edge_node(int t, int q, int &k, int &l) {
    const int e = t / q, s = t % q + 1;
    const int pm1 = q + 1;
    if (e == 0) { k = 0; l = s; }
    else if (e == 1) { k = pm1; l = s; }
    else if (e == 2) { k = s; l = 0; }
    else { k = s; l = pm1; }
}

struct LeafInfo {
    int p, q, n, n4, nbd, m, r, C, LDC;
    double sx, sy;
    const double *D, *D2, *coef, *f;
    int flags;  // bit 0: c12 != 0, bit 1: c1 != 0, bit 2: c2 != 0
};

// Workspace layout of one leaf: M = [A_ii | zero pad to n4 | -A_ib | f_I],
// row-major, ld LDC (a multiple of 4).
__device__ LeafInfo leaf_info(const CondenseParams &P, int leaf) {
    LeafInfo L;
    L.p = P.lt.p[leaf];
    L.q = L.p - 2;
    L.n = L.q * L.q;
    L.n4 = (L.n + 3) & ~3;
    L.nbd = 4 * L.q;
    L.m = P.m;
    L.r = L.nbd + L.m;
    L.C = L.n4 + L.r;
    L.LDC = (L.C + 3) & ~3;
    const double *box = P.lt.box + 4 * (long long)leaf;
    L.sx = 2.0 / box[2];
    L.sy = 2.0 / box[3];
    L.D = P.dt.dmat + P.dt.doff[L.p];
    L.D2 = L.D + L.p * L.p;
    L.coef = P.coef + 6 * P.lt.o_p2[leaf];
    L.f = (P.f != nullptr && P.m > 0) ? P.f + P.lt.o_p2[leaf] * P.m : nullptr;
    L.flags = 0;
    return L;
}

// Which optional operator terms are present on this leaf (block-uniform).
__device__ int leaf_flags(const LeafInfo &L) {
    const int p2 = L.p * L.p;
    int a = 0, b = 0, c = 0;
    for (int e = threadIdx.x; e < p2; e += NT) {
        a |= L.coef[p2 + e] != 0.0;
        b |= L.coef[3 * p2 + e] != 0.0;
        c |= L.coef[4 * p2 + e] != 0.0;
    }
    a = __syncthreads_or(a);
    b = __syncthreads_or(b);
    c = __syncthreads_or(c);
    return (a ? 1 : 0) | (b ? 2 : 0) | (c ? 4 : 0);
}

// Collocation operator entry A[(i,j),(k,l)] of
//   -(c11 u_xx + 2 c12 u_xy + c22 u_yy + c1 u_x + c2 u_y) - kappa^2 b u.
__device__ __forceinline__ double op_entry(const LeafInfo &L, int i, int j, int k, int l,
                                           double c11, double c12, double c22, double c1,
                                           double c2, double b, double kappa2) {
    const int p = L.p;
    double v = 0.0;
    if (l == j) v += c11 * L.sx * L.sx * L.D2[i * p + k] + c1 * L.sx * L.D[i * p + k];
    if (k == i) v += c22 * L.sy * L.sy * L.D2[j * p + l] + c2 * L.sy * L.D[j * p + l];
    if (L.flags & 1) v += 2.0 * c12 * L.sx * L.sy * L.D[i * p + k] * L.D[j * p + l];
    v = -v;
    if (k == i && l == j) v -= kappa2 * b;
    return v;
}

// M (row-major, ld LDC) <- [A_ii | 0 | -A_ib | f_I].  Entries that are
// structurally zero (no shared grid line, c12 == 0) are written without
// any FP64 arithmetic.
template <typename T>
__device__ void assemble(T *__restrict__ M, const LeafInfo &L, double kappa2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = L.p, q = L.q, p2 = p * p, nA = L.n4 + L.nbd;
    const bool dense = (L.flags & 1) != 0;
    for (int rr = warp; rr < L.n; rr += NWARP) {
        const int i = rr / q + 1, j = rr % q + 1, node = i * p + j;
        const double c11 = L.coef[node], c12 = L.coef[p2 + node], c22 = L.coef[2 * p2 + node];
        const double c1 = L.coef[3 * p2 + node], c2 = L.coef[4 * p2 + node];
        const double b = L.coef[5 * p2 + node];
        T *row = M + (long long)rr * L.LDC;
        for (int c = lane; c < L.C; c += 32) {
            T val = T(0);
            if (c < L.n || (c >= L.n4 && c < nA)) {
                int k, l;
                if (c < L.n) { k = c / q + 1; l = c % q + 1; }
                else edge_node(c - L.n4, q, k, l);
                if (dense || k == i || l == j) {
                    double v = op_entry(L, i, j, k, l, c11, c12, c22, c1, c2, b, kappa2);
                    val = (T)(c >= L.n4 ? -v : v);
                }
            } else if (c >= nA && L.f) {
                val = (T)L.f[(long long)node * L.m + (c - nA)];
            }
            row[c] = val;
        }
    }
}

// R = B - A_ii X in FP64, applied matrix-free: for column c the grid
// function holds X[:, c] at the interior nodes, the unit vector of edge node
// c (c < n_b) or zero (c >= n_b) on the edges, zero at the corners; B is 0
// for c < n_b (the -A_ib e_c term is inside A applied to that grid) and f_I
// otherwise.  Written to M[:, n + c] in the working type.
template <typename T>
__device__ void residual(T *__restrict__ M, const double *__restrict__ X, const LeafInfo &L,
                         double kappa2) {
    const int p = L.p, q = L.q, p2 = p * p, r = L.r, nbd = L.nbd;
    const double sxx = L.sx * L.sx, syy = L.sy * L.sy, sxy = L.sx * L.sy;
    for (long long e = threadIdx.x; e < (long long)L.n * r; e += NT) {
        const int rr = (int)(e / r), c = (int)(e % r);
        const int i = rr / q + 1, j = rr % q + 1, node = i * p + j;
        auto U = [&](int k, int l) -> double {
            if (k >= 1 && k <= q && l >= 1 && l <= q) return X[(long long)((k - 1) * q + (l - 1)) * r + c];
            if (c >= nbd) return 0.0;
            if ((k == 0 || k == p - 1) && (l == 0 || l == p - 1)) return 0.0;
            const int bi = (k == 0) ? (l - 1) : (k == p - 1) ? (q + l - 1) : (l == 0) ? (2 * q + k - 1) : (3 * q + k - 1);
            return bi == c ? 1.0 : 0.0;
        };
        double ux2 = 0.0, ux1 = 0.0, uy2 = 0.0, uy1 = 0.0, uxy = 0.0;
        const double *Di = L.D + i * p, *D2i = L.D2 + i * p;
        const double *Dj = L.D + j * p, *D2j = L.D2 + j * p;
        for (int k = 0; k < p; ++k) {
            const double u = U(k, j);
            ux2 = fma(D2i[k], u, ux2);
            if (L.flags & 2) ux1 = fma(Di[k], u, ux1);
        }
        for (int l = 0; l < p; ++l) {
            const double u = U(i, l);
            uy2 = fma(D2j[l], u, uy2);
            if (L.flags & 4) uy1 = fma(Dj[l], u, uy1);
        }
        if (L.flags & 1) {
            for (int k = 0; k < p; ++k) {
                double s = 0.0;
                for (int l = 0; l < p; ++l) s = fma(Dj[l], U(k, l), s);
                uxy = fma(Di[k], s, uxy);
            }
        }
        const double c11 = L.coef[node], c12 = L.coef[p2 + node], c22 = L.coef[2 * p2 + node];
        const double c1 = L.coef[3 * p2 + node], c2 = L.coef[4 * p2 + node], b = L.coef[5 * p2 + node];
        const double Au = -(c11 * sxx * ux2 + 2.0 * c12 * sxy * uxy + c22 * syy * uy2 + c1 * L.sx * ux1 +
                            c2 * L.sy * uy1) - kappa2 * b * U(i, j);
        const double Bv = (c >= nbd && L.f) ? L.f[(long long)node * L.m + (c - nbd)] : 0.0;
        M[(long long)rr * L.LDC + L.n4 + c] = (T)(Bv - Au);
    }
}

// S, W from X (FP64 values, row-major, ld ldx); T and h by the DtN rows:
// the outward normal derivative at edge node a is a combination of the
// nodes on the grid line through it (Section 2: flux on element boundaries).
template <typename XT>
__device__ void write_outputs(const CondenseParams &P, int leaf, const LeafInfo &L,
                              const XT *__restrict__ X, int ldx) {
    const int q = L.q, p = L.p, n = L.n, nbd = L.nbd, m = L.m, r = L.r;
    if (P.S) {
        double *S = P.S + P.lt.o_sb[leaf];
        for (long long e = threadIdx.x; e < (long long)n * nbd; e += NT) {
            const int i = (int)(e / nbd), b = (int)(e % nbd);
            S[e] = (double)X[(long long)i * ldx + b];
        }
    }
    if (P.W && m > 0) {
        double *W = P.W + P.lt.o_ni[leaf] * m;
        for (long long e = threadIdx.x; e < (long long)n * m; e += NT) {
            const int i = (int)(e / m), c = (int)(e % m);
            W[e] = (double)X[(long long)i * ldx + nbd + c];
        }
    }
    double *Tm = P.T + P.lt.o_bb[leaf];
    double *hm = (m > 0 && P.h) ? P.h + P.lt.o_nb[leaf] * m : nullptr;
    for (int e = threadIdx.x; e < nbd * r; e += NT) {
        const int a = e / r, b = e % r;
        const int edge = a / q, s = a % q;
        const bool far = (edge & 1);              // E or N: derivative row p-1
        const double sgn = far ? 1.0 : -1.0;
        const double scl = sgn * ((edge < 2) ? L.sx : L.sy);
        const double *Drow = L.D + (far ? (p - 1) * p : 0);
        double acc = 0.0;
        if (edge < 2) {
            for (int k = 1; k <= q; ++k) acc = fma(Drow[k], (double)X[(long long)((k - 1) * q + s) * ldx + b], acc);
        } else {
            for (int l = 1; l <= q; ++l) acc = fma(Drow[l], (double)X[(long long)(s * q + (l - 1)) * ldx + b], acc);
        }
        acc *= scl;
        if (b < nbd) {
            const int opp = (edge ^ 1) * q + s;   // edge node on the same line, other side
            if (b == a) acc += scl * Drow[far ? p - 1 : 0];
            if (b == opp) acc += scl * Drow[far ? 0 : p - 1];
            Tm[(long long)a * nbd + b] = acc;
        } else if (hm) {
            hm[(long long)a * m + (b - nbd)] = acc;
        }
    }
}

template <typename T, int NB, bool MIXED>
__global__ void __launch_bounds__(NT, 4) condense_kernel(CondenseParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem<T> sm = carve<T, NB>(smem_raw, P.blk.ldp);
    const int ldp = P.blk.ldp;
    unsigned char *slot = P.work + (long long)blockIdx.x * P.slot_bytes;
    T *M = (T *)slot;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(P.queue, 1);
            sm.misc[0] = t < P.n_leaves ? P.lt.order[t] : -1;
            sm.misc[1] = 0;
        }
        __syncthreads();
        const int leaf = sm.misc[0];
        if (leaf < 0) break;
        LeafInfo L = leaf_info(P, leaf);
        L.flags = leaf_flags(L);
        assemble<T>(M, L, P.kappa2);
        __syncthreads();
        if constexpr (!MIXED) {
            lu_solve<T, NB>(M, L.LDC, L.n, L.n4, L.C, true, nullptr, ldp, sm);
            write_outputs<T>(P, leaf, L, M + L.n4, L.LDC);
            __syncthreads();
            if (threadIdx.x == 0) P.info[leaf] = sm.misc[1];
        } else {
            const long long mbytes = (((long long)L.n * L.LDC * (long long)sizeof(T)) + 255) & ~255LL;
            double *X = (double *)(slot + mbytes);
            int *piv_g = (int *)(X + (long long)L.n * L.r);
            lu_solve<T, NB>(M, L.LDC, L.n, L.n4, L.C, true, piv_g, ldp, sm);
            for (long long e = threadIdx.x; e < (long long)L.n * L.r; e += NT) {
                const int i = (int)(e / L.r), c = (int)(e % L.r);
                X[e] = (double)M[(long long)i * L.LDC + L.n4 + c];
            }
            __syncthreads();
            int status = sm.misc[1];
            if (status == 0 && P.kmax > 0) {
                int it = 0;
                bool done = false;
                while (!done && it < P.kmax) {
                    residual<T>(M, X, L, P.kappa2);
                    __syncthreads();
                    lu_solve<T, NB>(M, L.LDC, L.n, L.n4, L.C, false, piv_g, ldp, sm);
                    int bad = 0;
                    for (int c = threadIdx.x; c < L.r; c += NT) {
                        double dmax = 0.0, xmax = 0.0;
                        for (int i = 0; i < L.n; ++i) {
                            const double d = (double)M[(long long)i * L.LDC + L.n4 + c];
                            const double x = X[(long long)i * L.r + c] + d;
                            X[(long long)i * L.r + c] = x;
                            dmax = fmax(dmax, fabs(d));
                            xmax = fmax(xmax, fabs(x));
                        }
                        if (!(dmax <= P.tol * xmax)) bad = 1;
                    }
                    bad = __syncthreads_or(bad);
                    ++it;
                    done = !bad;
                }
                if (!done) status = -it;
            }
            write_outputs<double>(P, leaf, L, X, L.r);
            __syncthreads();
            if (threadIdx.x == 0) P.info[leaf] = status;
        }
        __syncthreads();
    }
}

template <int NB>
__global__ void __launch_bounds__(NT) dense_solve_kernel(double *base, long long stride, int n, int n4, int C,
                                                       int LDC, int ldp, int *info) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem<double> sm = carve<double, NB>(smem_raw, ldp);
    if (threadIdx.x == 0) sm.misc[1] = 0;
    __syncthreads();
    lu_solve<double, NB>(base + (long long)blockIdx.x * stride, LDC, n, n4, C, true, nullptr, ldp, sm);
    if (threadIdx.x == 0 && info) info[blockIdx.x] = sm.misc[1];
}

// Node coordinates (Section 2 mesh): x0 + (1 - cos(i pi/(p-1))) hx/2.
__global__ void leaf_nodes_kernel(LeafTables lt, int n_leaves, double *xy) {
    const int leaf = blockIdx.x;
    if (leaf >= n_leaves) return;
    const int p = lt.p[leaf];
    const double *box = lt.box + 4LL * leaf;
    double *out = xy + 2 * lt.o_p2[leaf];
    const double inv = 1.0 / (p - 1);
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        out[e] = box[0] + (1.0 - cospi(i * inv)) * box[2] * 0.5;
        out[p * p + e] = box[1] + (1.0 - cospi(j * inv)) * box[3] * 0.5;
    }
}

}  // namespace

cudaError_t launch_leaf_nodes(const LeafTables &lt, int n_leaves, double *xy, cudaStream_t s) {
    leaf_nodes_kernel<<<n_leaves, 128, 0, s>>>(lt, n_leaves, xy);
    return cudaGetLastError();
}

namespace {

template <typename T, int NB>
size_t smem_of(int ldp) { return smem_bytes_for<T, NB>(ldp); }

template <typename K>
int occupancy(K kernel, size_t smem) {
    int nb = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, NT, smem) != cudaSuccess) return 0;
    return nb;
}

template <typename T, int NB, bool MIXED>
cudaError_t launch_one(const CondenseParams &prm, int grid, cudaStream_t s) {
    const size_t smem = smem_of<T, NB>(prm.blk.ldp);
    cudaError_t e = cudaFuncSetAttribute(condense_kernel<T, NB, MIXED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    condense_kernel<T, NB, MIXED><<<grid, NT, smem, s>>>(prm);
    return cudaGetLastError();
}

}  // namespace

// Panel width: the widest whose shared memory still allows three CTAs per
// SM (75 KB), never below 4.
LuBlocking choose_blocking(int prec, int nmax) {
    LuBlocking b;
    b.ldp = panel_ld(nmax);
    const bool dbl = prec == HPS_FP64;
    const int cands[3] = {dbl ? 16 : 32, dbl ? 8 : 16, dbl ? 4 : 8};
    b.nb_panel = cands[2];
    for (int nb : cands) {
        const size_t s = dbl ? (nb == 16 ? smem_of<double, 16>(b.ldp) : nb == 8 ? smem_of<double, 8>(b.ldp) : smem_of<double, 4>(b.ldp))
                             : (nb == 32 ? smem_of<float, 32>(b.ldp) : nb == 16 ? smem_of<float, 16>(b.ldp) : smem_of<float, 8>(b.ldp));
        if (s <= 75 * 1024) { b.nb_panel = nb; break; }
    }
    return b;
}

size_t condense_smem(int prec, const LuBlocking &b) {
    if (prec == HPS_FP64)
        return b.nb_panel == 16 ? smem_of<double, 16>(b.ldp) : b.nb_panel == 8 ? smem_of<double, 8>(b.ldp) : smem_of<double, 4>(b.ldp);
    return b.nb_panel == 32 ? smem_of<float, 32>(b.ldp) : b.nb_panel == 16 ? smem_of<float, 16>(b.ldp) : smem_of<float, 8>(b.ldp);
}

int condense_max_ctas_per_sm(int prec, const LuBlocking &b) {
    const size_t smem = condense_smem(prec, b);
    if (prec == HPS_FP64) {
        switch (b.nb_panel) {
            case 16: return occupancy(condense_kernel<double, 16, false>, smem);
            case 8: return occupancy(condense_kernel<double, 8, false>, smem);
            default: return occupancy(condense_kernel<double, 4, false>, smem);
        }
    }
    switch (b.nb_panel) {
        case 32: return occupancy(condense_kernel<float, 32, true>, smem);
        case 16: return occupancy(condense_kernel<float, 16, true>, smem);
        default: return occupancy(condense_kernel<float, 8, true>, smem);
    }
}

cudaError_t launch_condense(int prec, const CondenseParams &prm, int grid, cudaStream_t s) {
    if (prec == HPS_FP64) {
        switch (prm.blk.nb_panel) {
            case 16: return launch_one<double, 16, false>(prm, grid, s);
            case 8: return launch_one<double, 8, false>(prm, grid, s);
            default: return launch_one<double, 4, false>(prm, grid, s);
        }
    }
    switch (prm.blk.nb_panel) {
        case 32: return launch_one<float, 32, true>(prm, grid, s);
        case 16: return launch_one<float, 16, true>(prm, grid, s);
        default: return launch_one<float, 8, true>(prm, grid, s);
    }
}


cudaError_t launch_dense_solve(double *base, long long stride, int n, int n4, int C, int LDC, int batch,
                               int *info, cudaStream_t s) {
    const int ldp = panel_ld(n);
    size_t smem = smem_of<double, 16>(ldp);
    int nb = 16;
    if (smem > 100 * 1024) { nb = 8; smem = smem_of<double, 8>(ldp); }
    if (smem > 100 * 1024) { nb = 4; smem = smem_of<double, 4>(ldp); }
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e;
    switch (nb) {
        case 16:
            e = cudaFuncSetAttribute(dense_solve_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            dense_solve_kernel<16><<<batch, NT, smem, s>>>(base, stride, n, n4, C, LDC, ldp, info);
            break;
        case 8:
            e = cudaFuncSetAttribute(dense_solve_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            dense_solve_kernel<8><<<batch, NT, smem, s>>>(base, stride, n, n4, C, LDC, ldp, info);
            break;
        default:
            e = cudaFuncSetAttribute(dense_solve_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            dense_solve_kernel<4><<<batch, NT, smem, s>>>(base, stride, n, n4, C, LDC, ldp, info);
            break;
    }
    return cudaGetLastError();
}

}  // namespace hps
