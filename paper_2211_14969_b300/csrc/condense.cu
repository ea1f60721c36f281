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
#include <type_traits>

#include "hps_internal.cuh"

#include "dense_lu.cuh"

namespace hps {
namespace {

using namespace lu;

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

// float <-> double conversions done with integer operations on the bit
// patterns (IEEE 754 binary32 / binary64 layouts), so the refinement loop
// does not queue conversions behind the FP64 arithmetic.  Values outside the
// normal range take the conversion instruction.
__device__ __forceinline__ double f2d(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) {
        if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((unsigned long long)(u & 0x80000000u) << 32));
        return (double)f;
    }
    const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned long long ex = (unsigned long long)(e + (1023u - 127u)) << 52;
    const unsigned long long mt = (unsigned long long)(u & 0x7fffffu) << 29;
    return __longlong_as_double((long long)(s | ex | mt));
}

// double -> float keeping the leading 24 significant bits (truncation; a
// relative change below 2^-23 of a residual is immaterial to the correction
// it drives).
__device__ __forceinline__ float d2f_trunc(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    if ((u << 1) == 0ull) return __uint_as_float((unsigned)(u >> 32));
    const int e = (int)((u >> 52) & 0x7ffull) - 1023 + 127;
    if (e <= 0 || e >= 0xff) return (float)d;
    const unsigned s = (unsigned)(u >> 32) & 0x80000000u;
    const unsigned mt = (unsigned)((u >> 29) & 0x7fffffull);
    return __uint_as_float(s | ((unsigned)e << 23) | mt);
}


// Edge-node index of grid node (k, l) on the leaf boundary (not a corner).
__device__ __forceinline__ int edge_index(int k, int l, int p, int q) {
    return (k == 0) ? (l - 1) : (k == p - 1) ? (q + l - 1) : (l == 0) ? (2 * q + k - 1) : (3 * q + k - 1);
}

// M (row-major, ld LDC) <- [A_ii | 0 | -A_ib | f_I] for the operator
//   -(c11 u_xx + 2 c12 u_xy + c22 u_yy + c1 u_x + c2 u_y) - kappa^2 b u,
// one warp per row.  The row is zeroed, then only the nodes that share a
// grid line with the row's node are written (all nodes when c12 != 0).
// Corners are not unknowns: with c12 != 0 the mixed term reaches them, and a
// corner's value is the mean of the degree p-3 extrapolations along its two
// edges, so its entry is added to the edge columns with the weights
// l_l(-1)/2, l_l(+1)/2 that follow D*D in the tables.  The
// entries are formed in the working precision from per-row factors and the
// differentiation matrices held in that precision.  In FP32 the per-row
// factors are the coefficients (truncated to float on their bit patterns)
// times per-leaf float scales, which keeps the slow FP64 pipe out of the
// assembly; the FP32 matrix only drives the corrections, whose residuals
// use the FP64 factors.
template <typename T>
__device__ void assemble(T *__restrict__ M, const LeafInfo &L, const T *__restrict__ Dw, double kappa2) {
    using V = typename Vec<T>::type;
    constexpr int HV = Vec<T>::N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = L.p, q = L.q, p2 = p * p, nA = L.n4 + L.nbd;
    const T *D2w = Dw + p2;
    const bool dense = (L.flags & 1) != 0;
    // per-leaf scales of c11, c1, c22, c2, c12, b
    const T s11 = (T)(L.sx * L.sx), s1 = (T)L.sx, s22 = (T)(L.sy * L.sy), s2 = (T)L.sy;
    const T s12 = (T)(2.0 * L.sx * L.sy), sb = (T)kappa2;
    auto cvt = [](double v) -> T {
        if constexpr (sizeof(T) == 4) return d2f_trunc(v);
        else return v;
    };
    for (int rr = warp; rr < L.n; rr += NWARP) {
        const int i = rr / q + 1, j = rr - (i - 1) * q + 1, node = i * p + j;
        T ax2, ax1, ay2, ay1, axy, dg;
        if constexpr (sizeof(T) == 4) {
            ax2 = cvt(L.coef[node]) * s11;
            axy = cvt(L.coef[p2 + node]) * s12;
            ay2 = cvt(L.coef[2 * p2 + node]) * s22;
            ax1 = cvt(L.coef[3 * p2 + node]) * s1;
            ay1 = cvt(L.coef[4 * p2 + node]) * s2;
            dg = cvt(L.coef[5 * p2 + node]) * sb;
        } else {
            const double c11 = L.coef[node], c12 = L.coef[p2 + node], c22 = L.coef[2 * p2 + node];
            const double c1 = L.coef[3 * p2 + node], c2 = L.coef[4 * p2 + node];
            const double b = L.coef[5 * p2 + node];
            ax2 = c11 * L.sx * L.sx;
            ax1 = c1 * L.sx;
            ay2 = c22 * L.sy * L.sy;
            ay1 = c2 * L.sy;
            axy = 2.0 * c12 * L.sx * L.sy;
            dg = kappa2 * b;
        }
        T *row = M + (long long)rr * L.LDC;
        V zero;
        T *zp = (T *)&zero;
#pragma unroll
        for (int v = 0; v < HV; ++v) zp[v] = T(0);
        for (int c = lane * HV; c < L.LDC; c += 32 * HV) *(V *)(row + c) = zero;
        __syncwarp();
        // entry of column node (k, l): -(x-line + y-line + mixed) - kappa^2 b on the diagonal
        auto entry = [&](int k, int l) -> T {
            T v = T(0);
            if (l == j) v += ax2 * D2w[i * p + k] + ax1 * Dw[i * p + k];
            if (k == i) v += ay2 * D2w[j * p + l] + ay1 * Dw[j * p + l];
            if (dense) v += axy * Dw[i * p + k] * Dw[j * p + l];
            v = -v;
            if (k == i && l == j) v -= dg;
            return v;
        };
        const T *cw = D2w + p2;   // corner weights: [0, p) to the low end, [p, 2p) to the high end
        auto put = [&](int k, int l) {
            const bool bk = (k == 0 || k == p - 1), bl = (l == 0 || l == p - 1);
            if (bk && bl) return;  // corners are not unknowns
            T v = entry(k, l);
            if (!bk && !bl) {
                row[(k - 1) * q + (l - 1)] = v;
                return;
            }
            row[L.n4 + edge_index(k, l, p, q)] = -v;
        };
        if (!dense) {
            for (int t = lane; t < 2 * p; t += 32) {
                if (t < p) put(t, j);                       // the x-line through (i, j)
                else if (t - p != j) put(i, t - p);         // the y-line, diagonal already written
            }
        } else {
            // every node: the mixed term is the outer product of
            // a_k = axy Dx[i,k] and Dy[j,l]; the line terms and the corner
            // entries (mixed only) are formed once per line / per row
            const T *Dyj = Dw + j * p;
            const T a0 = axy * Dw[i * p], aP = axy * Dw[i * p + p - 1];
            const T c00 = -(a0 * Dyj[0]), c0P = -(a0 * Dyj[p - 1]);
            const T cP0 = -(aP * Dyj[0]), cPP = -(aP * Dyj[p - 1]);
            for (int k = 0; k < p; ++k) {
                const T ak = axy * Dw[i * p + k];
                const T xk = ax2 * D2w[i * p + k] + ax1 * Dw[i * p + k];   // x-line entry at column j
                const bool bk = (k == 0 || k == p - 1);
                for (int l = lane; l < p; l += 32) {
                    const bool bl = (l == 0 || l == p - 1);
                    if (bk && bl) continue;   // corners are not unknowns
                    T v = ak * Dyj[l];
                    if (l == j) v += xk;
                    if (k == i) v += ay2 * D2w[j * p + l] + ay1 * Dw[j * p + l];
                    v = -v;
                    if (k == i && l == j) v -= dg;
                    if (!bk && !bl) {
                        row[(k - 1) * q + (l - 1)] = v;
                    } else {
                        // the two corners at the ends of this node's edge
                        if (bk) v += cw[l] * (k == 0 ? c00 : cP0) + cw[p + l] * (k == 0 ? c0P : cPP);
                        else v += cw[k] * (l == 0 ? c00 : c0P) + cw[p + k] * (l == 0 ? cP0 : cPP);
                        row[L.n4 + edge_index(k, l, p, q)] = -v;
                    }
                }
            }
        }
        if (L.f)
            for (int c = lane; c < L.m; c += 32) row[nA + c] = cvt(L.f[(long long)node * L.m + c]);
    }
}

// Leaf solve: the right-hand sides f_I - A_ib u_b (M holds -A_ib from
// column n4 and f_I after it), moved to columns [n4, n4 + m); one warp per
// row, lanes over the columns.  Without the mixed term a row of A_ib has
// entries only at the four edge nodes on the row's two grid lines.
template <typename T>
__device__ void combine_rhs(T *__restrict__ M, const LeafInfo &L, const double *__restrict__ ub) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = L.q, nbd = L.nbd, m = L.m, n4 = L.n4;
    const bool dense = (L.flags & 1) != 0;
    auto cvt = [](double v) -> T {
        if constexpr (sizeof(T) == 4) return d2f_trunc(v);
        else return v;
    };
    constexpr int MAXV = 8;   // m <= 256
    for (int rr = warp; rr < L.n; rr += NWARP) {
        const int i = rr / q + 1, j = rr - (i - 1) * q + 1;
        const int e4[4] = {j - 1, q + j - 1, 2 * q + i - 1, 3 * q + i - 1};   // W, E, S, N
        T *row = M + (long long)rr * L.LDC;
        T v[MAXV];
#pragma unroll
        for (int t = 0; t < MAXV; ++t) {
            const int c = lane + 32 * t;
            v[t] = T(0);
            if (c < m) {
                T acc = row[n4 + nbd + c];
                if (dense) {
                    for (int e = 0; e < nbd; ++e) acc = fma(row[n4 + e], cvt(ub[(long long)e * m + c]), acc);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) acc = fma(row[n4 + e4[k]], cvt(ub[(long long)e4[k] * m + c]), acc);
                }
                v[t] = acc;
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < MAXV; ++t) {
            const int c = lane + 32 * t;
            if (c < m) row[n4 + c] = v[t];
        }
    }
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (a value carried as an unevaluated sum hi + lo of
// two floats), built from the error-free transformations TwoSum (Knuth) and
// FMA-based TwoProd (Dekker / Ogita-Rump-Oishi 2005).  About 48 significant
// bits, on the FP32 pipe.
// ---------------------------------------------------------------------------
struct DF { float hi, lo; };

// The _rn intrinsics are never contracted into FMAs, which would break the
// exactness these transformations rely on.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ DF df_from(double x) {
    DF r;
    r.hi = d2f_trunc(x);
    r.lo = d2f_trunc(x - f2d(r.hi));
    return r;
}

// acc += a * u (a, u double-float; acc kept as hi + lo, lo unnormalised)
__device__ __forceinline__ void df_mac(DF &acc, float ah, float al, float uh, float ul) {
    const float ph = __fmul_rn(ah, uh);
    float pe = fmaf(ah, uh, -ph);
    pe = fmaf(ah, ul, pe);
    pe = fmaf(al, uh, pe);
    float s, se;
    two_sum(acc.hi, ph, s, se);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(se, pe));
}

__device__ __forceinline__ DF df_norm(DF a) {
    DF r;
    r.hi = __fadd_rn(a.hi, a.lo);
    r.lo = __fsub_rn(a.lo, __fsub_rn(r.hi, a.hi));
    return r;
}

// Per interior node: the operator factors c11 sx^2, c1 sx, c22 sy^2, c2 sy,
// 2 c12 sx sy, kappa^2 b and the body loads are fixed for a leaf; they are
// formed once in FP64 and stored as double-float pairs (12 floats a node).
__device__ void node_factors(const LeafInfo &L, double kappa2, float *__restrict__ nf) {
    const int p = L.p, q = L.q, p2 = p * p;
    for (int rr = threadIdx.x; rr < L.n; rr += NT) {
        const int i = rr / q + 1, j = rr - (i - 1) * q + 1, node = i * p + j;
        const double v[6] = {L.coef[node] * L.sx * L.sx, L.coef[3 * p2 + node] * L.sx,
                             L.coef[2 * p2 + node] * L.sy * L.sy, L.coef[4 * p2 + node] * L.sy,
                             2.0 * L.coef[p2 + node] * L.sx * L.sy, kappa2 * L.coef[5 * p2 + node]};
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            const DF d = df_from(v[t]);
            nf[rr * 12 + 2 * t] = d.hi;
            nf[rr * 12 + 2 * t + 1] = d.lo;
        }
    }
}

// R = B - A_ii X (X as double-float pairs), applied matrix-free in
// double-float arithmetic: for column
// c the grid function holds X[:, c] at the interior nodes, the unit vector of
// edge node c (c < n_b) or zero (c >= n_b) on the edges, zero at the
// corners; B is 0 for c < n_b (the -A_ib e_c term is inside A applied to
// that grid) and f_I otherwise.  Written to M[:, n4 + c] in the working
// type.
// Columns go in chunks of cw, staged in shared memory as separate hi and lo
// float planes (Xh, Xl: n x cwp each, cwp = cw rounded up to 4, so a warp's
// 16-byte loads of consecutive column groups are consecutive); D and D^2 are
// staged as pairs in Dp.  Each thread takes one interior node and 4 columns;
// the x-line and y-line sums run in one loop, eight independent chains
// sharing the loop.  GENERAL adds the first-derivative and mixed terms
// (leaf_flags != 0); without them those terms are exactly zero and skipped.
// The mixed term sum_k Dx[i,k] sum_l Dy[j,l] u(k,l) reaches every node of
// the leaf; with sep it is evaluated in two passes per chunk, first
// V(k, j) = sum_l Dy[j,l] u(k,l) for every grid line k (hi and lo planes
// after Xl in shared memory, p q cwp each) and then sum_k Dx[i,k] V(k, j),
// 2 p^2 q instead of p^2 q^2 products per column; without sep (the caller's
// buffer has no room for V) every node sums all p^2 terms itself.
template <typename T, bool GENERAL, bool RESOLVE = false>
__device__ void residual(T *__restrict__ M, const float2 *__restrict__ X, const LeafInfo &L,
                         const float *__restrict__ Dh, const float *__restrict__ Dl,
                         const float *__restrict__ nf, float *__restrict__ Xs, float2 *__restrict__ Dp,
                         int cw_max, const double *__restrict__ ub = nullptr, bool sep = false) {
    constexpr int G = 4;
    const int p = L.p, q = L.q, r = L.r, nbd = L.nbd, n = L.n, p2 = p * p;
    for (int e = threadIdx.x; e < 2 * p2; e += NT) Dp[e] = make_float2(Dh[e], Dl[e]);
    const float2 *Dq = Dp, *D2q = Dp + p2;
    for (int c0 = 0; c0 < r; c0 += cw_max) {
        const int cw = min(cw_max, r - c0), cwp = (cw + 3) & ~3, ng = cwp / G;
        float *Xh = Xs, *Xl = Xs + (long long)n * cwp;
        for (int e = threadIdx.x; e < n * cwp; e += NT) {
            const int i = e / cwp, cc = e - i * cwp;
            float2 v = make_float2(0.0f, 0.0f);
            if (cc < cw) v = X[(long long)i * r + c0 + cc];
            Xh[e] = v.x;
            Xl[e] = v.y;
        }
        __syncthreads();
        // the grid function of chunk column cc at node (k, l): X inside, the
        // unit value of its edge node (condensation) or the edge data (leaf
        // solve) on the edges, the corner extrapolation at the corners
        auto U = [&](int k, int l, int cc) -> float2 {
            const int c = c0 + cc;
            if (k >= 1 && k <= q && l >= 1 && l <= q) {
                const int e = ((k - 1) * q + (l - 1)) * cwp + cc;
                return make_float2(Xh[e], Xl[e]);
            }
            if ((k == 0 || k == p - 1) && (l == 0 || l == p - 1)) {
                // the mean of the extrapolations along the corner's two edges
                const int o = 2 * p2;
                const int wl = (l == 0 ? 0 : p), wk = (k == 0 ? 0 : p);
                const int ev = (k == 0 ? 0 : q), eh = (l == 0 ? 2 * q : 3 * q);   // its W/E and S/N edge
                if constexpr (RESOLVE) {
                    DF acc = {0.0f, 0.0f};
                    for (int t2 = 1; t2 <= q; ++t2) {
                        const DF a = df_from(ub[(long long)(ev + t2 - 1) * L.m + c]);
                        const DF b = df_from(ub[(long long)(eh + t2 - 1) * L.m + c]);
                        df_mac(acc, Dh[o + wl + t2], Dl[o + wl + t2], a.hi, a.lo);
                        df_mac(acc, Dh[o + wk + t2], Dl[o + wk + t2], b.hi, b.lo);
                    }
                    acc = df_norm(acc);
                    return make_float2(acc.hi, acc.lo);
                }
                if (c >= ev && c < ev + q) return make_float2(Dh[o + wl + c - ev + 1], Dl[o + wl + c - ev + 1]);
                if (c >= eh && c < eh + q) return make_float2(Dh[o + wk + c - eh + 1], Dl[o + wk + c - eh + 1]);
                return make_float2(0.0f, 0.0f);
            }
            if constexpr (RESOLVE) {
                const DF e = df_from(ub[(long long)edge_index(k, l, p, q) * L.m + c]);
                return make_float2(e.hi, e.lo);
            }
            if (c >= nbd) return make_float2(0.0f, 0.0f);
            return make_float2(edge_index(k, l, p, q) == c ? 1.0f : 0.0f, 0.0f);
        };
        float *Vh = Xl + (long long)n * cwp, *Vl = Vh + (long long)p * q * cwp;
        const bool two_pass = GENERAL && sep && (L.flags & 1);
        if (two_pass) {
            for (int e = threadIdx.x; e < p * q * cw; e += NT) {
                const int cc = e % cw, kj = e / cw, k = kj / q, j = kj - k * q + 1;
                DF sk = {0.0f, 0.0f};
                for (int l = 0; l < p; ++l) {
                    const float2 u = U(k, l, cc);
                    df_mac(sk, Dq[j * p + l].x, Dq[j * p + l].y, u.x, u.y);
                }
                sk = df_norm(sk);
                Vh[(long long)kj * cwp + cc] = sk.hi;
                Vl[(long long)kj * cwp + cc] = sk.lo;
            }
            __syncthreads();
        }
        for (int w = threadIdx.x; w < n * ng; w += NT) {
            const int rr = w / ng, g = w - rr * ng;
            const int i = rr / q + 1, j = rr - (i - 1) * q + 1, node = i * p + j;
            DF ax2[G], ay2[G], ax1[G], ay1[G], axy[G];
#pragma unroll
            for (int t = 0; t < G; ++t) ax2[t] = ay2[t] = ax1[t] = ay1[t] = axy[t] = DF{0.0f, 0.0f};
            // x-line interior: nodes (k, j), k = 1..q, stride q rows;
            // y-line interior: nodes (i, l), l = 1..q, consecutive rows
            {
                const float *px = Xh + (j - 1) * cwp + g * G, *py = Xh + (i - 1) * q * cwp + g * G;
                const long long lo = (long long)n * cwp;
                const int sx = q * cwp, sy = cwp;
                for (int k = 1; k <= q; ++k, px += sx, py += sy) {
                    const float4 xh = *(const float4 *)px, xl = *(const float4 *)(px + lo);
                    const float4 yh = *(const float4 *)py, yl = *(const float4 *)(py + lo);
                    const float2 dx = D2q[i * p + k], dy = D2q[j * p + k];
                    df_mac(ax2[0], dx.x, dx.y, xh.x, xl.x);
                    df_mac(ay2[0], dy.x, dy.y, yh.x, yl.x);
                    df_mac(ax2[1], dx.x, dx.y, xh.y, xl.y);
                    df_mac(ay2[1], dy.x, dy.y, yh.y, yl.y);
                    df_mac(ax2[2], dx.x, dx.y, xh.z, xl.z);
                    df_mac(ay2[2], dy.x, dy.y, yh.z, yl.z);
                    df_mac(ax2[3], dx.x, dx.y, xh.w, xl.w);
                    df_mac(ay2[3], dy.x, dy.y, yh.w, yl.w);
                    if constexpr (GENERAL) {
                        if (L.flags & 2) {
                            const float2 d1 = Dq[i * p + k];
                            df_mac(ax1[0], d1.x, d1.y, xh.x, xl.x);
                            df_mac(ax1[1], d1.x, d1.y, xh.y, xl.y);
                            df_mac(ax1[2], d1.x, d1.y, xh.z, xl.z);
                            df_mac(ax1[3], d1.x, d1.y, xh.w, xl.w);
                        }
                        if (L.flags & 4) {
                            const float2 d1 = Dq[j * p + k];
                            df_mac(ay1[0], d1.x, d1.y, yh.x, yl.x);
                            df_mac(ay1[1], d1.x, d1.y, yh.y, yl.y);
                            df_mac(ay1[2], d1.x, d1.y, yh.z, yl.z);
                            df_mac(ay1[3], d1.x, d1.y, yh.w, yl.w);
                        }
                    }
                }
            }
            // edge nodes on the two lines carry the unit value of their column
            // (condensation) or the leaf's edge data (leaf solve)
            const int ew = j - 1, ee = q + j - 1, es = 2 * q + i - 1, en = 3 * q + i - 1;
            if constexpr (RESOLVE) {
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    const int c = c0 + g * G + t;
                    if (g * G + t >= cw) continue;
                    const DF uw = df_from(ub[(long long)ew * L.m + c]), ue = df_from(ub[(long long)ee * L.m + c]);
                    const DF us = df_from(ub[(long long)es * L.m + c]), un = df_from(ub[(long long)en * L.m + c]);
                    df_mac(ax2[t], D2q[i * p].x, D2q[i * p].y, uw.hi, uw.lo);
                    df_mac(ax2[t], D2q[i * p + p - 1].x, D2q[i * p + p - 1].y, ue.hi, ue.lo);
                    df_mac(ay2[t], D2q[j * p].x, D2q[j * p].y, us.hi, us.lo);
                    df_mac(ay2[t], D2q[j * p + p - 1].x, D2q[j * p + p - 1].y, un.hi, un.lo);
                    df_mac(ax1[t], Dq[i * p].x, Dq[i * p].y, uw.hi, uw.lo);
                    df_mac(ax1[t], Dq[i * p + p - 1].x, Dq[i * p + p - 1].y, ue.hi, ue.lo);
                    df_mac(ay1[t], Dq[j * p].x, Dq[j * p].y, us.hi, us.lo);
                    df_mac(ay1[t], Dq[j * p + p - 1].x, Dq[j * p + p - 1].y, un.hi, un.lo);
                }
            } else {
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    const int c = c0 + g * G + t;
                    if (c >= nbd) continue;
                    if (c == ew) { df_mac(ax2[t], D2q[i * p].x, D2q[i * p].y, 1.0f, 0.0f); df_mac(ax1[t], Dq[i * p].x, Dq[i * p].y, 1.0f, 0.0f); }
                    if (c == ee) { df_mac(ax2[t], D2q[i * p + p - 1].x, D2q[i * p + p - 1].y, 1.0f, 0.0f); df_mac(ax1[t], Dq[i * p + p - 1].x, Dq[i * p + p - 1].y, 1.0f, 0.0f); }
                    if (c == es) { df_mac(ay2[t], D2q[j * p].x, D2q[j * p].y, 1.0f, 0.0f); df_mac(ay1[t], Dq[j * p].x, Dq[j * p].y, 1.0f, 0.0f); }
                    if (c == en) { df_mac(ay2[t], D2q[j * p + p - 1].x, D2q[j * p + p - 1].y, 1.0f, 0.0f); df_mac(ay1[t], Dq[j * p + p - 1].x, Dq[j * p + p - 1].y, 1.0f, 0.0f); }
                }
            }
            if constexpr (GENERAL) {
                if (L.flags & 1) {   // mixed derivative: every node of the leaf
#pragma unroll
                    for (int t = 0; t < G; ++t) {
                        const int cc = g * G + t;
                        if (cc >= cw) continue;
                        if (two_pass) {
                            for (int k = 0; k < p; ++k) {
                                const long long v = ((long long)k * q + (j - 1)) * cwp + cc;
                                df_mac(axy[t], Dq[i * p + k].x, Dq[i * p + k].y, Vh[v], Vl[v]);
                            }
                            continue;
                        }
                        for (int k = 0; k < p; ++k) {
                            DF sk = {0.0f, 0.0f};
                            for (int l = 0; l < p; ++l) {
                                const float2 u = U(k, l, cc);
                                df_mac(sk, Dq[j * p + l].x, Dq[j * p + l].y, u.x, u.y);
                            }
                            sk = df_norm(sk);
                            df_mac(axy[t], Dq[i * p + k].x, Dq[i * p + k].y, sk.hi, sk.lo);
                        }
                    }
                }
            }
            // A u = -(a2x ux2 + a1x ux1 + a2y uy2 + a1y uy1 + axy uxy) - dg u_ij;
            // R = B - A u with B = f for load columns
            const float *f6 = nf + rr * 12;
            const float4 uh = *(const float4 *)(Xh + rr * cwp + g * G), ul = *(const float4 *)(Xl + rr * cwp + g * G);
            const float uhv[G] = {uh.x, uh.y, uh.z, uh.w}, ulv[G] = {ul.x, ul.y, ul.z, ul.w};
#pragma unroll
            for (int t = 0; t < G; ++t) {
                const int cc = g * G + t, c = c0 + cc;
                if (cc >= cw) continue;
                DF au = {0.0f, 0.0f};
                const DF t0 = df_norm(ax2[t]), t2 = df_norm(ay2[t]);
                df_mac(au, f6[0], f6[1], t0.hi, t0.lo);
                if constexpr (GENERAL) {
                    const DF t1 = df_norm(ax1[t]);
                    df_mac(au, f6[2], f6[3], t1.hi, t1.lo);
                }
                df_mac(au, f6[4], f6[5], t2.hi, t2.lo);
                if constexpr (GENERAL) {
                    const DF t3 = df_norm(ay1[t]), t4 = df_norm(axy[t]);
                    df_mac(au, f6[6], f6[7], t3.hi, t3.lo);
                    df_mac(au, f6[8], f6[9], t4.hi, t4.lo);
                }
                df_mac(au, f6[10], f6[11], uhv[t], ulv[t]);
                if ((RESOLVE || c >= nbd) && L.f) {
                    const DF b = df_from(L.f[(long long)node * L.m + (RESOLVE ? c : c - nbd)]);
                    float s2, se;
                    two_sum(au.hi, b.hi, s2, se);
                    au.hi = s2;
                    au.lo = __fadd_rn(au.lo, __fadd_rn(se, b.lo));
                }
                M[(long long)rr * L.LDC + L.n4 + c] = (T)__fadd_rn(au.hi, au.lo);
            }
        }
        __syncthreads();
    }
}

// S, W from X (FP64 values, row-major, ld ldx); T and h by the DtN rows:
// the outward normal derivative at edge node a is a combination of the
// nodes on the grid line through it (Section 2: flux on element boundaries).
// Rows by warp, columns by lane.
template <typename XT>
__device__ void write_outputs(const CondenseParams &P, int leaf, const LeafInfo &L,
                              const XT *__restrict__ X, int ldx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = L.q, p = L.p, n = L.n, nbd = L.nbd, m = L.m, r = L.r;
    double *S = P.S ? P.S + P.lt.o_sb[leaf] : nullptr;
    double *W = (P.W && m > 0) ? P.W + P.lt.o_ni[leaf] * m : nullptr;
    for (int i = warp; i < n; i += NWARP) {
        const XT *xr = X + (long long)i * ldx;
        if (S)
            for (int b = lane; b < nbd; b += 32) S[(long long)i * nbd + b] = (double)xr[b];
        if (W)
            for (int cc = lane; cc < m; cc += 32) W[(long long)i * m + cc] = (double)xr[nbd + cc];
    }
    double *Tm = P.T + P.lt.o_bb[leaf];
    double *hm = (m > 0 && P.h) ? P.h + P.lt.o_nb[leaf] * m : nullptr;
    for (int a = warp; a < nbd; a += NWARP) {
        const int edge = a / q, s = a - edge * q;
        const bool far = (edge & 1);              // E or N: derivative row p-1
        const double scl = (far ? 1.0 : -1.0) * ((edge < 2) ? L.sx : L.sy);
        const double *Drow = L.D + (far ? (p - 1) * p : 0);
        // interior nodes on the line: (k, s+1) for W/E, (s+1, l) for S/N
        const long long base = (edge < 2) ? s : (long long)s * q;
        const long long step = (edge < 2) ? q : 1;
        const int opp = (edge ^ 1) * q + s;   // edge node on the same line, other side
        for (int b = lane; b < r; b += 32) {
            double acc = 0.0;
            for (int k = 1; k <= q; ++k) acc = fma(Drow[k], (double)X[(base + (k - 1) * step) * ldx + b], acc);
            acc *= scl;
            if (b < nbd) {
                if (b == a) acc += scl * Drow[far ? p - 1 : 0];
                if (b == opp) acc += scl * Drow[far ? 0 : p - 1];
                Tm[(long long)a * nbd + b] = acc;
            } else if (hm) {
                hm[(long long)a * m + (b - nbd)] = acc;
            }
        }
    }
}

// The same outputs from the mixed path's iterate X (n x r double-float
// pairs): the DtN sums run in double-float arithmetic with D split into
// hi/lo floats (Dh, Dl), so the FP64 pipe only forms the final doubles.
__device__ void write_outputs_df(const CondenseParams &P, int leaf, const LeafInfo &L,
                                 const float2 *__restrict__ X, const float *__restrict__ Dh,
                                 const float *__restrict__ Dl) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = L.q, p = L.p, n = L.n, nbd = L.nbd, m = L.m, r = L.r;
    double *S = P.S ? P.S + P.lt.o_sb[leaf] : nullptr;
    double *W = (P.W && m > 0) ? P.W + P.lt.o_ni[leaf] * m : nullptr;
    {   // S and W: X row by row, eight loads in flight per thread
        const int nr = n * r;
        for (int e0 = threadIdx.x; e0 < nr; e0 += 8 * NT) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = e0 + u * NT < nr ? X[e0 + u * NT] : make_float2(0.0f, 0.0f);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * NT, i = e / r, b = e - i * r;
                if (e >= nr) continue;
                const double x = f2d(v[u].x) + f2d(v[u].y);
                if (b < nbd) {
                    if (S) S[(long long)i * nbd + b] = x;
                } else if (W) {
                    W[(long long)i * m + (b - nbd)] = x;
                }
            }
        }
    }
    double *Tm = P.T + P.lt.o_bb[leaf];
    double *hm = (m > 0 && P.h) ? P.h + P.lt.o_nb[leaf] * m : nullptr;
    for (int a = warp; a < nbd; a += NWARP) {
        const int edge = a / q, s = a - edge * q;
        const bool far = (edge & 1);              // E or N: derivative row p-1
        const double scl = (far ? 1.0 : -1.0) * ((edge < 2) ? L.sx : L.sy);
        const double *Drow = L.D + (far ? (p - 1) * p : 0);
        const float *Dhr = Dh + (far ? (p - 1) * p : 0), *Dlr = Dl + (far ? (p - 1) * p : 0);
        const long long base = (edge < 2) ? s : (long long)s * q;
        const long long step = (edge < 2) ? q : 1;
        const int opp = (edge ^ 1) * q + s;
        for (int b = lane; b < r; b += 32) {
            DF acc = {0.0f, 0.0f};
            for (int k = 1; k <= q; ++k) {
                const float2 x = X[(base + (k - 1) * step) * r + b];
                df_mac(acc, Dhr[k], Dlr[k], x.x, x.y);
            }
            double v = (f2d(acc.hi) + f2d(acc.lo)) * scl;
            if (b < nbd) {
                if (b == a) v += scl * Drow[far ? p - 1 : 0];
                if (b == opp) v += scl * Drow[far ? 0 : p - 1];
                Tm[(long long)a * nbd + b] = v;
            } else if (hm) {
                hm[(long long)a * m + (b - nbd)] = v;
            }
        }
    }
}

// Leaf solve output: u at every node [p*p][m]: interior nodes from the
// solution X (FP64 values, ld ldx, or double-float pairs), edge nodes from
// the given edge values, corners 0 (they are not unknowns).
template <typename XT>
__device__ __forceinline__ double x_value(const XT &x) {
    if constexpr (std::is_same<XT, float2>::value) return f2d(x.x) + f2d(x.y);
    else return (double)x;
}
template <typename XT>
__device__ void write_u(const CondenseParams &P, int leaf, const LeafInfo &L, const XT *__restrict__ X, int ldx,
                        const double *__restrict__ ub) {
    const int p = L.p, q = L.q, m = L.m;
    double *u = P.u + P.lt.o_p2[leaf] * m;
    for (int e = threadIdx.x; e < p * p * m; e += NT) {
        const int node = e / m, c = e - node * m, i = node / p, j = node - i * p;
        const bool bi = (i == 0 || i == p - 1), bj = (j == 0 || j == p - 1);
        double v = 0.0;
        if (bi != bj) v = ub[(long long)edge_index(i, j, p, q) * m + c];
        else if (!bi) v = x_value(X[(long long)((i - 1) * q + (j - 1)) * ldx + c]);
        u[e] = v;
    }
}

// X (n x r double-float pairs) += correction in M[:, n4..]; returns (block-uniform)
// whether every column's estimated error after this correction is <= tol.
// eta[c] holds the previous relative correction of column c (1 before the
// first); the estimate for linearly converging refinement is
// eta_k^2 / eta_{k-1}, and a column that stopped contracting never passes.
template <typename T>
__device__ bool refine_update(T *__restrict__ M, float2 *__restrict__ X, float *__restrict__ eta,
                              const LeafInfo &L, double tol, unsigned *colmax, bool allow_stop = true) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = L.r;
    for (int c = threadIdx.x; c < 2 * r; c += NT) colmax[c] = 0u;
    __syncthreads();
    constexpr int UB = 8;   // rows whose loads are all issued before the first is used
    for (int c0 = 0; c0 < r; c0 += 32) {
        const int c = c0 + lane;
        float dmax = 0.0f, xmax = 0.0f;
        if (c < r) {
            for (int i0 = warp; i0 < L.n; i0 += NWARP * UB) {
                float dv[UB];
                float2 xv[UB];
#pragma unroll
                for (int u = 0; u < UB; ++u) {
                    const int i = i0 + u * NWARP;
                    if (i < L.n) {
                        dv[u] = (float)M[(long long)i * L.LDC + L.n4 + c];
                        xv[u] = X[(long long)i * r + c];
                    }
                }
#pragma unroll
                for (int u = 0; u < UB; ++u) {
                    const int i = i0 + u * NWARP;
                    if (i >= L.n) continue;
                    const float d = dv[u];
                    const float2 x = xv[u];
                    float s, e;
                    two_sum(x.x, d, s, e);
                    const float lo = __fadd_rn(x.y, e);
                    const float hi = __fadd_rn(s, lo);   // renormalise: |lo| well below ulp(s)
                    X[(long long)i * r + c] = make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s)));
                    dmax = fmaxf(dmax, fabsf(d));
                    xmax = fmaxf(xmax, fabsf(hi));
                }
            }
            // non-negative floats order like their bit patterns; NaN maps high
            atomicMax(&colmax[c], dmax == dmax ? __float_as_uint(dmax) : 0x7f800000u);
            atomicMax(&colmax[r + c], __float_as_uint(xmax));
        }
    }
    __syncthreads();
    int bad = 0;
    for (int c = threadIdx.x; c < r; c += NT) {
        const float dmax = __uint_as_float(colmax[c]), xmax = __uint_as_float(colmax[r + c]);
        const float e_k = xmax > 0.0f ? dmax / xmax : (dmax > 0.0f ? 1.0f : 0.0f);
        const float e_prev = eta[c];
        const bool contracting = e_k < e_prev || e_k == 0.0f;
        const double est = e_prev > 0.0f ? (double)e_k * (double)e_k / (double)e_prev : 0.0;
        if (!(contracting && est <= tol)) bad = 1;
        eta[c] = e_k;
    }
    return __syncthreads_or(bad) == 0 && allow_stop;
}

// Column maxima |R| of the residual just written to M[:, n4 .. n4 + r),
// into colmax (shared memory, r unsigned: bit patterns of non-negative
// floats, NaN high); eight rows' loads in flight per thread.  A pass of its
// own, so the residual's register budget is untouched.
template <typename T>
__device__ void residual_colmax(const T *__restrict__ M, const LeafInfo &L, unsigned *colmax) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, r = L.r;
    for (int c = threadIdx.x; c < r; c += NT) colmax[c] = 0u;
    __syncthreads();
    constexpr int UB = 8;
    for (int c0 = 0; c0 < r; c0 += 32) {
        const int c = c0 + lane;
        if (c >= r) continue;
        float mx = 0.0f;
        for (int i0 = warp; i0 < L.n; i0 += NWARP * UB) {
            float v[UB];
#pragma unroll
            for (int u = 0; u < UB; ++u) {
                const int i = i0 + u * NWARP;
                v[u] = i < L.n ? fabsf((float)M[(long long)i * L.LDC + L.n4 + c]) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < UB; ++u) mx = fmaxf(mx, v[u]);
        }
        atomicMax(&colmax[c], mx == mx ? __float_as_uint(mx) : 0x7f800000u);
    }
    __syncthreads();
}

// The first correction's stop: X_1's error estimated per column from the
// true residuals as eta_1 |R_1| / |R_0| (the correction eta_1 measured X_0's
// error; the residual ratio measures how much of it the correction
// removed).  Block-uniform; rn1 holds |R_1| per column (float bit patterns,
// shared memory), rn0 |R_0| (the slot).
__device__ bool residual_ratio_ok(const unsigned *rn1, const float *rn0, const float *eta, int r, double tol) {
    int bad = 0;
    for (int c = threadIdx.x; c < r; c += NT) {
        const float r1 = __uint_as_float(rn1[c]), r0 = rn0[c];
        const double est = r0 > 0.0f ? (double)eta[c] * (double)r1 / (double)r0 : 0.0;
        if (!(est <= tol)) bad = 1;
    }
    return __syncthreads_or(bad) == 0;
}

// Offset of the tensor-core operand buffers behind the LU's shared memory.
__host__ __device__ inline size_t tc_smem_offset(size_t lu_bytes) { return (lu_bytes + 1023) & ~(size_t)1023; }

template <typename T, int NB, bool MIXED, int TCK = 0, bool RSTOP = false>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 4) condense_kernel(CondenseParams P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const Smem<T> sm = carve<T, NB>(smem_raw, P.blk.ldp);
    const int ldp = P.blk.ldp;
    constexpr bool INV = use_inverses<T, NB, TCK>();   // L11 inverses kept (FP32 path)
    unsigned char *slot = P.work + (long long)blockIdx.x * P.slot_bytes;
    T *M = (T *)slot;
    tc::TcState tcs{};
    const tc::TcState *tsp = nullptr;
    if constexpr (TCK != 0) {
        unsigned char *b = smem_raw + tc_smem_offset(smem_bytes_for<T, NB>(ldp));
        constexpr int EB = tc::In<TCK>::BYTES;
        tcs.a_hi = b;
        tcs.a_lo = b + tc::TM * NB * EB;
        tcs.b_hi = b + 2 * tc::TM * NB * EB;
        tcs.b_lo = tcs.b_hi + tc::TN * NB * EB;
        unsigned char *tail = b + tc::operand_bytes<TCK>(NB);
        tcs.mbar = (uint64_t *)tail;
        tcs.tmem = (uint32_t *)(tail + 8);
        tcs.phase = (uint32_t *)(tail + 12);
        tcs.err = (int *)(tail + 16);
        tc::tmem_alloc(tcs);
        tsp = &tcs;
    }
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(P.queue, 1);
            sm.misc[0] = t < P.n_leaves ? P.lt.order[t] : -1;
            sm.misc[1] = 0;
        }
        __syncthreads();
        const int leaf = sm.misc[0];
        if (leaf < 0) break;
        if constexpr (TCK != 0) {
            if (threadIdx.x == 0) *tcs.err = 0;
        }
        LeafInfo L = leaf_info(P, leaf);
        L.flags = leaf_flags(L);
        const double *ubl = P.ub ? P.ub + P.lt.o_nb[leaf] * L.m : nullptr;   // leaf solve: edge values
        const T *Dw = (const T *)(sizeof(T) == 4 ? (const void *)P.dt.dmat32 : (const void *)P.dt.dmat) + P.dt.doff[L.p];
        assemble<T>(M, L, Dw, P.kappa2);
        __syncthreads();
        if (ubl) {   // one right-hand side per load: f_I - A_ib u_b
            combine_rhs<T>(M, L, ubl);
            __syncthreads();
            L.r = L.m;
            L.C = L.n4 + L.m;
        }
        if constexpr (!MIXED) {
            lu_solve<T, NB>(M, L.LDC, L.n, L.n4, L.C, true, nullptr, ldp, sm);
            if (ubl) write_u<T>(P, leaf, L, M + L.n4, L.LDC, ubl);
            else write_outputs<T>(P, leaf, L, M + L.n4, L.LDC);
            __syncthreads();
            if (threadIdx.x == 0) P.info[leaf] = sm.misc[1];
        } else {
            const long long mbytes = (((long long)L.n * L.LDC * (long long)sizeof(T)) + 255) & ~255LL;
            float2 *X = (float2 *)(slot + mbytes);                // iterate, double-float pairs
            int *perm_g = (int *)(X + (long long)L.n * L.r);   // 3 NB ints per panel
            lu_solve<T, NB, TCK, INV>(M, L.LDC, L.n, L.n4, L.C, true, perm_g, ldp, sm, tsp);
            float *eta = (float *)(perm_g + 3 * (L.n + 64));
            // column max |R_0| at eta + round64(r), then 12 floats per interior node
            float *nf = eta + 2 * ((L.r + 63) & ~63);
            const float *Dhi = P.dt.dmat32 + P.dt.doff[L.p], *Dlo = P.dt.dmat_lo + P.dt.doff[L.p];
            node_factors(L, P.kappa2, nf);
            // residual column chunk: as many FP64 columns as the panel and
            // chunk buffers hold (they are idle between eliminations)
            // the D/D^2 pairs take the front of the buffer, X chunks the rest
            const int dpairs = 2 * L.p * L.p;
            const long long buf2 = (long long)((size_t)NB * (ldp + Cfg<T, NB>::CH) * sizeof(T) / sizeof(float2)) - dpairs;
            const int xs_cap = (int)(buf2 / L.n);
            int xs_cols = xs_cap >= 16 ? 16 : xs_cap >= 8 ? 8 : 4;
            // with the mixed term, the grid-line sums V take p q pairs a column
            // beside X's n when the buffer holds at least 4 such columns
            bool sep = false;
            if (L.flags & 1) {
                const int cap2 = (int)(buf2 / (L.n + L.p * L.q));
                if (cap2 >= 4) {
                    sep = true;
                    xs_cols = cap2 >= 16 ? 16 : cap2 >= 8 ? 8 : 4;
                }
            }
            {   // X = the FP32 solution; eight loads in flight per thread
                const int nr = L.n * L.r;
                for (int e0 = threadIdx.x; e0 < nr; e0 += 8 * NT) {
                    float v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int e = e0 + u * NT, i = e / L.r, c = e - i * L.r;
                        v[u] = e < nr ? (float)M[(long long)i * L.LDC + L.n4 + c] : 0.0f;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (e0 + u * NT < nr) X[e0 + u * NT] = make_float2(v[u], 0.0f);
                }
            }
            for (int c = threadIdx.x; c < L.r; c += NT) eta[c] = 1.0f;
            __syncthreads();
            int status = sm.misc[1];
            if constexpr (TCK != 0) {
                if (*tcs.err) status = HPS_INFO_TC_TIMEOUT;   // a tensor-core wait timed out
            }
            if (status == 0 && P.kmax > 0) {
                int it = 0;
                bool done = false;
                while (!done && it < P.kmax) {
                    float *xs = (float *)((float2 *)sm.Ps + 2 * L.p * L.p);
                    if (ubl) residual<T, true, true>(M, X, L, Dhi, Dlo, nf, xs, (float2 *)sm.Ps, xs_cols, ubl, sep);
                    else if (L.flags) residual<T, true>(M, X, L, Dhi, Dlo, nf, xs, (float2 *)sm.Ps, xs_cols, nullptr, sep);
                    else residual<T, false>(M, X, L, Dhi, Dlo, nf, xs, (float2 *)sm.Ps, xs_cols);
                    __syncthreads();
                    // the first two residuals' column maxima: after the first
                    // correction the true residual decides whether X_1 is
                    // already good enough
                    if (RSTOP && it <= 1) {
                        unsigned *cm = (unsigned *)sm.Us;   // idle between the residual and the replay
                        float *rn0 = eta + ((L.r + 63) & ~63);
                        residual_colmax<T>(M, L, cm);
                        if (it == 0) {
                            for (int c = threadIdx.x; c < L.r; c += NT) rn0[c] = __uint_as_float(cm[c]);
                            __syncthreads();
                        } else if (residual_ratio_ok(cm, rn0, eta, L.r, P.tol)) {
                            done = true;
                            break;
                        }
                    }
                    lu_solve<T, NB, 0, INV>(M, L.LDC, L.n, L.n4, L.C, false, perm_g, ldp, sm);
                    // the correction-ratio estimate stops from the second correction on
                    done = refine_update<T>(M, X, eta, L, P.tol, (unsigned *)sm.Us, !RSTOP || it >= 1 || P.kmax == 1);
                    ++it;
                }
                if (!done) status = -it;
            }
            if (status < 0 && status != HPS_INFO_TC_TIMEOUT && P.fallback) {
                // Refinement did not converge (a leaf too ill-conditioned for
                // FP32 factors): condense it again in FP64 in the same slot,
                // with the double-precision blocking of half the panel width
                // (its shared memory fits inside this kernel's).
                const Smem<double> sd = carve<double, NB / 2>(smem_raw, ldp);
                double *M64 = (double *)slot;
                __syncthreads();
                assemble<double>(M64, L, P.dt.dmat + P.dt.doff[L.p], P.kappa2);
                if (threadIdx.x == 0) sd.misc[1] = 0;
                __syncthreads();
                if (ubl) {
                    combine_rhs<double>(M64, L, ubl);
                    __syncthreads();
                }
                lu_solve<double, NB / 2>(M64, L.LDC, L.n, L.n4, L.C, true, nullptr, ldp, sd);
                if (ubl) write_u<double>(P, leaf, L, M64 + L.n4, L.LDC, ubl);
                else write_outputs<double>(P, leaf, L, M64 + L.n4, L.LDC);
                status = sd.misc[1];
                if (threadIdx.x == 0) atomicAdd(P.fallbacks, 1);
            } else if (ubl) {
                write_u<float2>(P, leaf, L, X, L.r, ubl);
            } else {
                write_outputs_df(P, leaf, L, X, P.dt.dmat32 + P.dt.doff[L.p], P.dt.dmat_lo + P.dt.doff[L.p]);
            }
            __syncthreads();
            if (threadIdx.x == 0) P.info[leaf] = status;
        }
        __syncthreads();
    }
    if constexpr (TCK != 0) tc::tmem_free(tcs);
}

// ---------------------------------------------------------------------------
// Impedance-to-impedance leaf maps.  The leaf system with the impedance
// condition (N u)_a + i eta u_a = f_a at every edge node a (the PDE rows at
// the interior nodes as for the DtN maps, corners folded into the edge
// columns) is complex; it is assembled in real form over the unknowns
// [Re u_i (n) | Re u_b (nb) | Im u_i (n) | Im u_b (nb)] with the rows in the
// same order (PDE, impedance; real parts, then imaginary parts) and solved
// by the FP64 blocked LU for nb unit incoming-data columns and the m body
// loads.  Y = X_re + i X_im; R = I - 2 i eta Y_b, h = -2 i eta uf_b.
// ---------------------------------------------------------------------------

struct ItiInfo {
    int N, R2, n4, C, LDC;   // N = n + nb unknowns per part, R2 = 2N real rows
};

__device__ ItiInfo iti_info(const LeafInfo &L) {
    ItiInfo I;
    I.N = L.n + L.nbd;
    I.R2 = 2 * I.N;
    I.n4 = (I.R2 + 3) & ~3;
    I.C = I.n4 + L.nbd + L.m;
    I.LDC = (I.C + 3) & ~3;
    return I;
}

// One warp per real row: zero the row, then its entries.
__device__ void assemble_iti(double *__restrict__ M, const LeafInfo &L, const ItiInfo &I, const double *__restrict__ D,
                             double kappa2, double eta) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = L.p, q = L.q, p2 = p * p, n = L.n, N = I.N;
    const double *D2 = D + p2, *cw = D2 + p2;
    const bool dense = (L.flags & 1) != 0;
    for (int row = warp; row < I.R2; row += NWARP) {
        double *r = M + (long long)row * I.LDC;
        for (int c = lane * 2; c < I.LDC; c += 64) *(double2 *)(r + c) = make_double2(0.0, 0.0);
        __syncwarp();
        const int part = row / N, rr = row - part * N;   // part 0: real rows, 1: imaginary rows
        const int off = part * N;                         // their unknowns' columns
        if (rr < n) {
            // PDE at interior node (i, j): A_ii into [off, off + n), A_ib into [off + n, off + N)
            const int i = rr / q + 1, j = rr - (i - 1) * q + 1, node = i * p + j;
            const double ax2 = L.coef[node] * L.sx * L.sx, ax1 = L.coef[3 * p2 + node] * L.sx;
            const double ay2 = L.coef[2 * p2 + node] * L.sy * L.sy, ay1 = L.coef[4 * p2 + node] * L.sy;
            const double axy = 2.0 * L.coef[p2 + node] * L.sx * L.sy, dg = kappa2 * L.coef[5 * p2 + node];
            // corner values of the mixed term: corner (k, l) with k, l in {0, p-1}
            const double c00 = -(axy * D[i * p] * D[j * p]), c0P = -(axy * D[i * p] * D[j * p + p - 1]);
            const double cP0 = -(axy * D[i * p + p - 1] * D[j * p]), cPP = -(axy * D[i * p + p - 1] * D[j * p + p - 1]);
            for (int e = lane; e < p2; e += 32) {
                const int k = e / p, l = e - k * p;
                const bool bk = (k == 0 || k == p - 1), bl = (l == 0 || l == p - 1);
                if (bk && bl) continue;                                   // corners are not unknowns
                if (!dense && k != i && l != j) continue;                 // off the two grid lines: zero
                double v = 0.0;
                if (l == j) v += ax2 * D2[i * p + k] + ax1 * D[i * p + k];
                if (k == i) v += ay2 * D2[j * p + l] + ay1 * D[j * p + l];
                if (dense) v += axy * D[i * p + k] * D[j * p + l];
                v = -v;
                if (k == i && l == j) v -= dg;
                if (!bk && !bl) {
                    r[off + (k - 1) * q + (l - 1)] = v;
                } else {
                    if (dense) {   // the corners at the ends of this edge node's edge (mean extrapolation)
                        if (bk) v += cw[l] * (k == 0 ? c00 : cP0) + cw[p + l] * (k == 0 ? c0P : cPP);
                        else v += cw[k] * (l == 0 ? c00 : c0P) + cw[p + k] * (l == 0 ? cP0 : cPP);
                    }
                    r[off + n + edge_index(k, l, p, q)] = v;
                }
            }
            if (part == 0 && L.f)
                for (int c = lane; c < L.m; c += 32) r[I.n4 + L.nbd + c] = L.f[(long long)node * L.m + c];
        } else {
            // impedance condition at edge node a: the outward normal derivative
            // along the grid line through a, plus i eta u_a
            const int a = rr - n, edge = a / q, s = a - edge * q;
            const bool far = (edge & 1);
            const double scl = (far ? 1.0 : -1.0) * ((edge < 2) ? L.sx : L.sy);
            const double *Drow = D + (far ? (p - 1) * p : 0);
            const int lo = (edge < 2) ? s : 2 * q + s, hi = (edge < 2) ? q + s : 3 * q + s;   // W/S and E/N ends
            for (int k = lane; k < p; k += 32) {
                const double v = scl * Drow[k];
                if (k == 0) r[off + n + lo] += v;
                else if (k == p - 1) r[off + n + hi] += v;
                else r[off + ((edge < 2) ? (k - 1) * q + s : s * q + (k - 1))] = v;
            }
            __syncwarp();
            if (lane == 0) {
                if (part == 0) {
                    r[N + n + a] = -eta;           // Re: (N u_re) - eta u_im = Re f
                    r[I.n4 + a] = 1.0;             // unit incoming data, real
                } else {
                    r[n + a] = eta;                // Im: (N u_im) + eta u_re = Im f
                }
            }
        }
    }
}

// Outputs from X = M[:, n4 ..] (2N x (nb + m)), complex interleaved (re, im):
// R [nb][nb], h [nb][m], and for the interior recovery Y_i [n][nb], uf_i [n][m].
__device__ void write_iti(const CondenseParams &P, int leaf, const LeafInfo &L, const ItiInfo &I,
                          const double *__restrict__ M) {
    const int n = L.n, nb = L.nbd, m = L.m, N = I.N;
    const double e2 = 2.0 * P.eta;
    double *R = P.T + 2 * P.lt.o_bb[leaf];
    double *h = (m > 0 && P.h) ? P.h + 2 * P.lt.o_nb[leaf] * m : nullptr;
    double *Y = P.S ? P.S + 2 * P.lt.o_sb[leaf] : nullptr;
    double *uf = (m > 0 && P.W) ? P.W + 2 * P.lt.o_ni[leaf] * m : nullptr;
    const int cols = nb + m;
    for (int e = threadIdx.x; e < N * cols; e += NT) {
        const int row = e / cols, c = e - row * cols;
        const double xr = M[(long long)row * I.LDC + I.n4 + c];
        const double xi = M[(long long)(N + row) * I.LDC + I.n4 + c];
        if (row >= n) {
            const int a = row - n;
            if (c < nb) {   // R = I - 2 i eta Y_b
                R[2 * ((long long)a * nb + c)] = (a == c ? 1.0 : 0.0) + e2 * xi;
                R[2 * ((long long)a * nb + c) + 1] = -e2 * xr;
            } else if (h) {
                h[2 * ((long long)a * m + c - nb)] = e2 * xi;
                h[2 * ((long long)a * m + c - nb) + 1] = -e2 * xr;
            }
        } else if (c < nb) {
            if (Y) {
                Y[2 * ((long long)row * nb + c)] = xr;
                Y[2 * ((long long)row * nb + c) + 1] = xi;
            }
        } else if (uf) {
            uf[2 * ((long long)row * m + c - nb)] = xr;
            uf[2 * ((long long)row * m + c - nb) + 1] = xi;
        }
    }
}

template <int NB>
__global__ void __launch_bounds__(NT, 4) iti_kernel(CondenseParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem<double> sm = carve<double, NB>(smem_raw, P.blk.ldp);
    double *M = (double *)(P.work + (long long)blockIdx.x * P.slot_bytes);
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
        const ItiInfo I = iti_info(L);
        assemble_iti(M, L, I, P.dt.dmat + P.dt.doff[L.p], P.kappa2, P.eta);
        __syncthreads();
        lu_solve<double, NB>(M, I.LDC, I.R2, I.n4, I.C, true, nullptr, P.blk.ldp, sm);
        write_iti(P, leaf, L, I, M);
        __syncthreads();
        if (threadIdx.x == 0) P.info[leaf] = sm.misc[1];
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

// u_i = S u_b + W per leaf (the stored-operator leaf solve), leaves of any
// order: one CTA per leaf, one thread per output node and column.
__global__ void __launch_bounds__(NT) leaf_recover_all_kernel(LeafTables lt, int m, const double *__restrict__ S,
                                                             const double *__restrict__ W,
                                                             const double *__restrict__ ub, double *__restrict__ u) {
    const int leaf = blockIdx.x, p = lt.p[leaf], q = p - 2, nbd = 4 * q;
    const double *Sl = S + lt.o_sb[leaf];
    const double *Wl = W ? W + lt.o_ni[leaf] * m : nullptr;
    const double *ul = ub + lt.o_nb[leaf] * m;
    double *uo = u + lt.o_p2[leaf] * m;
    for (int e = threadIdx.x; e < p * p * m; e += NT) {
        const int node = e / m, c = e - node * m, i = node / p, j = node - i * p;
        const bool bi = (i == 0 || i == p - 1), bj = (j == 0 || j == p - 1);
        double v = 0.0;
        if (bi != bj) {
            v = ul[(long long)edge_index(i, j, p, q) * m + c];
        } else if (!bi) {
            const int r = (i - 1) * q + (j - 1);
            v = Wl ? Wl[(long long)r * m + c] : 0.0;
            const double *Sr = Sl + (long long)r * nbd;
            for (int b = 0; b < nbd; ++b) v = fma(Sr[b], ul[(long long)b * m + c], v);
        }
        uo[e] = v;
    }
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

cudaError_t launch_leaf_recover_all(const LeafTables &lt, int n_leaves, int m, const double *S, const double *W,
                                    const double *ub, double *u, cudaStream_t s) {
    leaf_recover_all_kernel<<<n_leaves, NT, 0, s>>>(lt, m, S, W, ub, u);
    return cudaGetLastError();
}

cudaError_t launch_leaf_nodes(const LeafTables &lt, int n_leaves, double *xy, cudaStream_t s) {
    leaf_nodes_kernel<<<n_leaves, 128, 0, s>>>(lt, n_leaves, xy);
    return cudaGetLastError();
}

namespace {

template <typename T, int NB>
size_t smem_of(int ldp) { return smem_bytes_for<T, NB>(ldp, use_inverses<T, NB, 0>()); }

template <typename K>
int occupancy(K kernel, size_t smem) {
    int nb = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, NT, smem) != cudaSuccess) return 0;
    return nb;
}

template <typename T, int NB, int TCK>
size_t kernel_smem(int ldp) {
    if constexpr (TCK == 0) return smem_of<T, NB>(ldp);
    else return tc_smem_offset(smem_bytes_for<T, NB>(ldp)) + tc::operand_bytes<TCK>(NB) + 64;
}

template <typename T, int NB, bool MIXED, int TCK = 0, bool RSTOP = false>
cudaError_t launch_kernel(const CondenseParams &prm, int grid, cudaStream_t s) {
    const size_t smem = kernel_smem<T, NB, TCK>(prm.blk.ldp);
    cudaError_t e = cudaFuncSetAttribute(condense_kernel<T, NB, MIXED, TCK, RSTOP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    condense_kernel<T, NB, MIXED, TCK, RSTOP><<<grid, NT, smem, s>>>(prm);
    return cudaGetLastError();
}

// The first correction's true-residual stop is its own instantiation of the
// FP32 CUDA-core kernel (hps_set_refine_stop), so the default kernels'
// register allocation does not carry its code.
template <typename T, int NB, bool MIXED, int TCK = 0>
cudaError_t launch_one(const CondenseParams &prm, int grid, cudaStream_t s) {
    if constexpr (MIXED && TCK == 0) {
        if (prm.residual_stop) return launch_kernel<T, NB, MIXED, TCK, true>(prm, grid, s);
    }
    return launch_kernel<T, NB, MIXED, TCK, false>(prm, grid, s);
}

}  // namespace

// Panel width: the widest whose shared memory still allows three CTAs per
// SM (75 KB), never below 4.  The mixed path also stages, between
// eliminations, the differentiation pairs and 4 columns of the FP64 iterate
// in the panel and chunk buffers; the panel is widened until they fit.
LuBlocking choose_blocking(int prec, int nmax, int pmax) {
    LuBlocking b;
    b.ldp = panel_ld(nmax);
    const bool dbl = prec == HPS_FP64;
    const int cands[3] = {dbl ? 16 : 32, dbl ? 8 : 16, dbl ? 4 : 8};
    auto bytes = [&](int nb) {
        return dbl ? (nb == 16 ? smem_of<double, 16>(b.ldp) : nb == 8 ? smem_of<double, 8>(b.ldp) : smem_of<double, 4>(b.ldp))
                   : (nb == 32 ? smem_of<float, 32>(b.ldp) : nb == 16 ? smem_of<float, 16>(b.ldp) : smem_of<float, 8>(b.ldp));
    };
    int pick = 2;
    for (int t = 0; t < 3; ++t)
        if (bytes(cands[t]) <= 75 * 1024) { pick = t; break; }
    if (!dbl) {
        const size_t need = (size_t)(2 * pmax * pmax + 4 * nmax) * 8;
        while (pick > 0 && (size_t)cands[pick] * (b.ldp + 64) * sizeof(float) < need) --pick;
    }
    b.nb_panel = cands[pick];
    return b;
}

size_t condense_smem(int prec, const LuBlocking &b) {
    const int nb = b.nb_panel;
    switch (prec) {
        case HPS_FP64:
            return nb == 16 ? smem_of<double, 16>(b.ldp) : nb == 8 ? smem_of<double, 8>(b.ldp) : smem_of<double, 4>(b.ldp);
        case HPS_MIXED_TF32:
            return nb == 32 ? kernel_smem<float, 32, tc::KIND_TF32>(b.ldp)
                 : nb == 16 ? kernel_smem<float, 16, tc::KIND_TF32>(b.ldp) : kernel_smem<float, 8, tc::KIND_TF32>(b.ldp);
        case HPS_MIXED_BF16:
            return nb == 32 ? kernel_smem<float, 32, tc::KIND_BF16>(b.ldp)
                 : nb == 16 ? kernel_smem<float, 16, tc::KIND_BF16>(b.ldp) : kernel_smem<float, 8, tc::KIND_BF16>(b.ldp);
        default:
            return nb == 32 ? smem_of<float, 32>(b.ldp) : nb == 16 ? smem_of<float, 16>(b.ldp) : smem_of<float, 8>(b.ldp);
    }
}

int condense_max_ctas_per_sm(int prec, const LuBlocking &b) {
    const size_t smem = condense_smem(prec, b);
    const int nb = b.nb_panel;
    switch (prec) {
        case HPS_FP64:
            return nb == 16 ? occupancy(condense_kernel<double, 16, false>, smem)
                 : nb == 8 ? occupancy(condense_kernel<double, 8, false>, smem) : occupancy(condense_kernel<double, 4, false>, smem);
        case HPS_MIXED_TF32:
            return nb == 32 ? occupancy(condense_kernel<float, 32, true, tc::KIND_TF32>, smem)
                 : nb == 16 ? occupancy(condense_kernel<float, 16, true, tc::KIND_TF32>, smem)
                            : occupancy(condense_kernel<float, 8, true, tc::KIND_TF32>, smem);
        case HPS_MIXED_BF16:
            return nb == 32 ? occupancy(condense_kernel<float, 32, true, tc::KIND_BF16>, smem)
                 : nb == 16 ? occupancy(condense_kernel<float, 16, true, tc::KIND_BF16>, smem)
                            : occupancy(condense_kernel<float, 8, true, tc::KIND_BF16>, smem);
        default:
            return nb == 32 ? occupancy(condense_kernel<float, 32, true>, smem)
                 : nb == 16 ? occupancy(condense_kernel<float, 16, true>, smem) : occupancy(condense_kernel<float, 8, true>, smem);
    }
}

LuBlocking iti_blocking(int nmax_real) {
    LuBlocking b;
    b.ldp = panel_ld(nmax_real);
    b.nb_panel = smem_of<double, 16>(b.ldp) <= 75 * 1024 ? 16 : smem_of<double, 8>(b.ldp) <= 75 * 1024 ? 8 : 4;
    return b;
}

static size_t iti_smem(const LuBlocking &b) {
    return b.nb_panel == 16 ? smem_of<double, 16>(b.ldp) : b.nb_panel == 8 ? smem_of<double, 8>(b.ldp)
                                                                            : smem_of<double, 4>(b.ldp);
}

int iti_max_ctas_per_sm(const LuBlocking &b) {
    const size_t smem = iti_smem(b);
    return b.nb_panel == 16 ? occupancy(iti_kernel<16>, smem)
         : b.nb_panel == 8 ? occupancy(iti_kernel<8>, smem) : occupancy(iti_kernel<4>, smem);
}

cudaError_t launch_iti(const CondenseParams &prm, int grid, cudaStream_t s) {
    const size_t smem = iti_smem(prm.blk);
    cudaError_t e = cudaSuccess;
    switch (prm.blk.nb_panel) {
        case 16:
            e = cudaFuncSetAttribute(iti_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) iti_kernel<16><<<grid, NT, smem, s>>>(prm);
            break;
        case 8:
            e = cudaFuncSetAttribute(iti_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) iti_kernel<8><<<grid, NT, smem, s>>>(prm);
            break;
        default:
            e = cudaFuncSetAttribute(iti_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) iti_kernel<4><<<grid, NT, smem, s>>>(prm);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_condense(int prec, const CondenseParams &prm, int grid, cudaStream_t s) {
    const int nb = prm.blk.nb_panel;
    switch (prec) {
        case HPS_FP64:
            return nb == 16 ? launch_one<double, 16, false>(prm, grid, s)
                 : nb == 8 ? launch_one<double, 8, false>(prm, grid, s) : launch_one<double, 4, false>(prm, grid, s);
        case HPS_MIXED_TF32:
            return nb == 32 ? launch_one<float, 32, true, tc::KIND_TF32>(prm, grid, s)
                 : nb == 16 ? launch_one<float, 16, true, tc::KIND_TF32>(prm, grid, s)
                            : launch_one<float, 8, true, tc::KIND_TF32>(prm, grid, s);
        case HPS_MIXED_BF16:
            return nb == 32 ? launch_one<float, 32, true, tc::KIND_BF16>(prm, grid, s)
                 : nb == 16 ? launch_one<float, 16, true, tc::KIND_BF16>(prm, grid, s)
                            : launch_one<float, 8, true, tc::KIND_BF16>(prm, grid, s);
        default:
            return nb == 32 ? launch_one<float, 32, true>(prm, grid, s)
                 : nb == 16 ? launch_one<float, 16, true>(prm, grid, s) : launch_one<float, 8, true>(prm, grid, s);
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
