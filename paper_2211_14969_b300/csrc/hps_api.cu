// C ABI of libhps (declared in include/hps.h): plan construction, argument
// checking, workspace management and the launch sequence of every call.
// All numerical work runs in the kernels of condense.cu and merge.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <array>
#include <vector>

#include "hps.h"
#include "hps_internal.cuh"
#include "merge.cuh"

using namespace hps;

namespace {

// Message of the last failed call without a plan (hps_build_leaves,
// hps_condense_noalloc) on this host thread: thread_local, so threads that
// fail at the same time do not race on it.
thread_local std::string g_build_error;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t want) {
        if (bytes >= want) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) bytes = want;
        else p = nullptr;
        return e;
    }
};

struct Level {
    MergeLevelDev dev{};
    DevBuf maps, aug, th, u, info, piv, u3, oz;
};

long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

constexpr int kMaxTimed = 4096;

// Chebyshev differentiation matrix on the p Chebyshev-Gauss-Lobatto points
// of [-1, 1] in increasing order, from the barycentric weights
// w_k = (-1)^k (1/2 at the ends): D_ij = (w_j / w_i) / (t_i - t_j), with the
// node differences taken in the product form 2 sin(pi(i+j)/2N) sin(pi(i-j)/2N)
// (Don & Solomonoff 1997) and the diagonal from the zero row sum.
void chebyshev_matrix(int p, std::vector<double> &D) {
    const int N = p - 1;
    const double pi = 3.14159265358979323846;
    std::vector<double> w(p);
    for (int k = 0; k < p; ++k) w[k] = ((k & 1) ? -1.0 : 1.0) * ((k == 0 || k == N) ? 0.5 : 1.0);
    D.assign((size_t)p * p, 0.0);
    for (int i = 0; i < p; ++i) {
        double s = 0.0;
        for (int j = 0; j < p; ++j) {
            if (j == i) continue;
            const double diff = 2.0 * std::sin(pi * (i + j) / (2.0 * N)) * std::sin(pi * (i - j) / (2.0 * N));
            const double v = (w[j] / w[i]) / diff;
            D[(size_t)i * p + j] = v;
            s += v;
        }
        D[(size_t)i * p + i] = -s;
    }
}

// Corner extrapolation weights of order p: the Lagrange basis of the p - 2
// interior Chebyshev points t_1..t_q of [-1, 1] evaluated at the ends,
// halved (a corner is the mean of the extrapolations along its two edges):
// ce[l] = l_l(-1) / 2 and ce[p + l] = l_l(+1) / 2 for l = 1..q, zero at
// l = 0 and p - 1.  Barycentric form with w_k = 1 / prod_{m != k}(t_k - t_m).
void corner_weights(int p, std::vector<double> &ce) {
    const int q = p - 2, N = p - 1;
    const double pi = 3.14159265358979323846;
    std::vector<double> t(q), w(q);
    for (int k = 0; k < q; ++k) t[k] = -std::cos(pi * (k + 1) / N);
    for (int k = 0; k < q; ++k) {
        double d = 1.0;
        for (int m = 0; m < q; ++m)
            if (m != k) d *= (t[k] - t[m]);
        w[k] = 1.0 / d;
    }
    ce.assign(2 * (size_t)p, 0.0);
    for (int side = 0; side < 2; ++side) {
        const double s = side ? 1.0 : -1.0;
        double den = 0.0;
        for (int k = 0; k < q; ++k) den += w[k] / (s - t[k]);
        for (int k = 0; k < q; ++k) ce[(size_t)side * p + k + 1] = 0.5 * (w[k] / (s - t[k])) / den;
    }
}

}  // namespace

namespace hps {
// Sets the text returned by hps_last_error(NULL) (calls without a plan).
void set_global_error(const std::string &msg) { g_build_error = msg; }
}  // namespace hps

struct hps_plan {
    int n_leaves = 0;
    double kappa = 0.0;
    std::vector<int> p;
    std::vector<double> box;
    int pmin = 0, pmax = 0;
    bool uniform = true;
    std::vector<long long> o_p2, o_ni, o_nb, o_sb, o_bb;
    DevBuf tables, work;
    int *d_p = nullptr, *d_order = nullptr, *d_doff = nullptr, *d_queue = nullptr;
    double *d_box = nullptr, *d_dmat = nullptr;
    float *d_dmat32 = nullptr, *d_dmat_lo = nullptr;
    long long *d_off = nullptr;  // o_p2, o_ni, o_nb, o_sb, o_bb back to back
    int device = 0, sms = 0;
    bool timing = false;
    std::vector<cudaEvent_t> ev;  // pairs around each recorded kernel
    int n_timed = 0;
    int launches = 0;
    int forced_nb[2] = {0, 0};   // per path (FP64, mixed); 0 = automatic
    int fallback = 1;            // mixed path: re-condense non-converged leaves in FP64
    int residual_stop = 0;       // mixed path: first correction's stop on the true residuals (off by default)
    cudaStream_t last_stream = nullptr;
    // merge tree
    std::vector<Level> levels;
    DevBuf u_leaf;
    int merge_nx = 0, merge_ny = 0, merge_m = -1;
    int merge_wx0 = 1, merge_wy0 = 1;   // unit box of the last merge (1 x 1: the leaves)
    bool merged = false;
    // SlabLU: the slabs' [T | h], the interfaces' solved systems, solve scratch
    DevBuf slab_th, slab_aug, slab_piv, slab_info, slab_tmp;
    int slab_nx = 0, slab_ny = 0, slab_s = 0, slab_m = -1;
    bool slabbed = false;
    int split_below = -1;  // levels with fewer merges solve Z over many CTAs; -1: the SM count
    int merge_tensor = 1;  // large merge products on the tensor cores (ozaki.cu); 2: SlabLU's interface solves too
    DevBuf oz_err;         // their timeout flag
    DevBuf slab_oz;        // tensor-core scratch of SlabLU's interface solves
    SplitAux split_aux{nullptr, nullptr, nullptr};   // look-ahead stream and events, made on first use
    // hps_condense_host: device copies of the inputs and outputs, the chunk
    // work-queue orders and counters, two more streams and their events
    DevBuf hstage, horder;
    std::vector<int> horder_host;         // kept alive until its upload completes
    cudaStream_t hs_comp = nullptr, hs_h2d = nullptr, hs_d2h = nullptr;
    std::vector<cudaEvent_t> hev;
    std::string err;

    hps_status fail(hps_status s, const std::string &msg) {
        err = msg;
        return s;
    }
    hps_status cuda_fail(cudaError_t e, const char *where) {
        err = std::string(where) + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? HPS_ERR_OOM : HPS_ERR_CUDA;
    }
    // event pair i (created on first use)
    cudaEvent_t *event_pair(int i) {
        while ((int)ev.size() < 2 * (i + 1)) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            ev.push_back(e);
        }
        return &ev[2 * i];
    }
    LeafTables leaf_tables() const {
        LeafTables t;
        t.p = d_p;
        t.box = d_box;
        const long long nl = n_leaves;
        t.o_p2 = d_off;
        t.o_ni = d_off + nl;
        t.o_nb = d_off + 2 * nl;
        t.o_sb = d_off + 3 * nl;
        t.o_bb = d_off + 4 * nl;
        t.order = d_order;
        return t;
    }
};

extern "C" {

int hps_version(void) { return 105; }

const char *hps_last_error(const hps_plan *plan) {
    if (plan == nullptr) return g_build_error.c_str();
    return plan->err.c_str();
}

hps_status hps_build_leaves(const hps_leaf_desc *desc, hps_plan **out, hps_stream stream) {
    if (out == nullptr) {
        g_build_error = "hps_build_leaves: out is NULL";
        return HPS_ERR_ARG;
    }
    *out = nullptr;
    if (desc == nullptr || desc->n_leaves < 1 || desc->p == nullptr || desc->box == nullptr) {
        g_build_error = "hps_build_leaves: empty or NULL leaf description";
        return HPS_ERR_ARG;
    }
    if (!std::isfinite(desc->kappa)) {
        g_build_error = "hps_build_leaves: kappa is not finite";
        return HPS_ERR_ARG;
    }
    const int nl = desc->n_leaves;
    for (int l = 0; l < nl; ++l) {
        const int p = desc->p[l];
        const double *b = desc->box + 4LL * l;
        if (p < HPS_PMIN || p > HPS_PMAX) {
            g_build_error = "hps_build_leaves: leaf " + std::to_string(l) + " has p = " + std::to_string(p) +
                            " outside [" + std::to_string(HPS_PMIN) + ", " + std::to_string(HPS_PMAX) + "]";
            return HPS_ERR_ARG;
        }
        if (!(b[2] > 0.0) || !(b[3] > 0.0) || !std::isfinite(b[0]) || !std::isfinite(b[1]) ||
            !std::isfinite(b[2]) || !std::isfinite(b[3])) {
            g_build_error = "hps_build_leaves: leaf " + std::to_string(l) + " has an invalid box";
            return HPS_ERR_ARG;
        }
    }
    hps_plan *P = new hps_plan();
    P->n_leaves = nl;
    P->kappa = desc->kappa;
    P->p.assign(desc->p, desc->p + nl);
    P->box.assign(desc->box, desc->box + 4LL * nl);
    P->pmin = *std::min_element(P->p.begin(), P->p.end());
    P->pmax = *std::max_element(P->p.begin(), P->p.end());
    P->uniform = P->pmin == P->pmax;
    P->o_p2.resize(nl); P->o_ni.resize(nl); P->o_nb.resize(nl); P->o_sb.resize(nl); P->o_bb.resize(nl);
    long long a = 0, b = 0, c = 0, d = 0, e = 0;
    for (int l = 0; l < nl; ++l) {
        const long long p = P->p[l], q = p - 2;
        P->o_p2[l] = a; P->o_ni[l] = b; P->o_nb[l] = c; P->o_sb[l] = d; P->o_bb[l] = e;
        a += p * p; b += q * q; c += 4 * q; d += q * q * 4 * q; e += 16 * q * q;
    }
    // largest leaves first; equal orders keep their index order
    std::vector<int> order(nl);
    for (int l = 0; l < nl; ++l) order[l] = l;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return P->p[x] > P->p[y]; });
    // Chebyshev tables for every order present
    std::vector<int> doff(HPS_PMAX + 1, -1);
    std::vector<double> dmat;
    for (int p = HPS_PMIN; p <= HPS_PMAX; ++p) {
        if (std::find(P->p.begin(), P->p.end(), p) == P->p.end()) continue;
        std::vector<double> D;
        chebyshev_matrix(p, D);
        doff[p] = (int)dmat.size();
        dmat.insert(dmat.end(), D.begin(), D.end());
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) {
                double s = 0.0;
                for (int k = 0; k < p; ++k) s += D[(size_t)i * p + k] * D[(size_t)k * p + j];
                dmat.push_back(s);
            }
        std::vector<double> ce;
        corner_weights(p, ce);
        dmat.insert(dmat.end(), ce.begin(), ce.end());
    }
    cudaError_t err = cudaGetDevice(&P->device);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, P->device);
    if (err != cudaSuccess) {
        g_build_error = std::string("hps_build_leaves: ") + cudaGetErrorString(err);
        delete P;
        return HPS_ERR_CUDA;
    }
    // one allocation for all tables
    const size_t sz_p = round_up(sizeof(int) * nl, 256), sz_box = round_up(sizeof(double) * 4 * nl, 256);
    const size_t sz_off = round_up(sizeof(long long) * 5 * nl, 256), sz_ord = sz_p;
    const size_t sz_doff = round_up(sizeof(int) * (HPS_PMAX + 1), 256);
    const size_t sz_dmat = round_up(sizeof(double) * std::max<size_t>(dmat.size(), 1), 256);
    const size_t sz_q = 256;
    const size_t sz_dmat32 = round_up(sizeof(float) * std::max<size_t>(dmat.size(), 1), 256);
    std::vector<float> dmat32(dmat.begin(), dmat.end()), dmat_lo(dmat.size());
    for (size_t k = 0; k < dmat.size(); ++k) dmat_lo[k] = (float)(dmat[k] - (double)dmat32[k]);
    err = P->tables.ensure(sz_p + sz_box + sz_off + sz_ord + sz_doff + sz_dmat + 2 * sz_dmat32 + sz_q);
    if (err != cudaSuccess) {
        g_build_error = std::string("hps_build_leaves: cudaMalloc: ") + cudaGetErrorString(err);
        delete P;
        return err == cudaErrorMemoryAllocation ? HPS_ERR_OOM : HPS_ERR_CUDA;
    }
    unsigned char *base = (unsigned char *)P->tables.p;
    P->d_p = (int *)base; base += sz_p;
    P->d_box = (double *)base; base += sz_box;
    P->d_off = (long long *)base; base += sz_off;
    P->d_order = (int *)base; base += sz_ord;
    P->d_doff = (int *)base; base += sz_doff;
    P->d_dmat = (double *)base; base += sz_dmat;
    P->d_dmat32 = (float *)base; base += sz_dmat32;
    P->d_dmat_lo = (float *)base; base += sz_dmat32;
    P->d_queue = (int *)base;
    std::vector<long long> off;
    off.reserve(5LL * nl);
    for (auto *v : {&P->o_p2, &P->o_ni, &P->o_nb, &P->o_sb, &P->o_bb}) off.insert(off.end(), v->begin(), v->end());
    cudaStream_t s = (cudaStream_t)stream;
    err = cudaMemcpyAsync(P->d_p, P->p.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(P->d_box, P->box.data(), sizeof(double) * 4 * nl, cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(P->d_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(P->d_order, order.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(P->d_doff, doff.data(), sizeof(int) * doff.size(), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess && !dmat.empty())
        err = cudaMemcpyAsync(P->d_dmat, dmat.data(), sizeof(double) * dmat.size(), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess && !dmat32.empty())
        err = cudaMemcpyAsync(P->d_dmat32, dmat32.data(), sizeof(float) * dmat32.size(), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess && !dmat_lo.empty())
        err = cudaMemcpyAsync(P->d_dmat_lo, dmat_lo.data(), sizeof(float) * dmat_lo.size(), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);  // host staging vectors die here
    if (err != cudaSuccess) {
        g_build_error = std::string("hps_build_leaves: upload: ") + cudaGetErrorString(err);
        delete P;
        return HPS_ERR_CUDA;
    }
    *out = P;
    return HPS_OK;
}

hps_status hps_leaf_nodes(const hps_plan *plan, double *d_xy, hps_stream stream) {
    if (plan == nullptr || d_xy == nullptr) return HPS_ERR_ARG;
    cudaError_t e = launch_leaf_nodes(plan->leaf_tables(), plan->n_leaves, d_xy, (cudaStream_t)stream);
    if (e != cudaSuccess) return const_cast<hps_plan *>(plan)->cuda_fail(e, "hps_leaf_nodes");
    return HPS_OK;
}

// One launch over a subset of the leaves (hps_condense_host): its work-queue
// order, length and counter, and which half of a doubled workspace its CTAs
// use (so two consecutive subsets can run concurrently).
struct CondenseChunk {
    const int *order;
    int n;
    int *queue;
    int half;
};

// The condensation launch, shared by hps_condense, hps_leaf_resolve
// (d_ub != nullptr: leaf solve, outputs in d_u) and hps_condense_host (ck:
// one subset of the leaves; the caller resets the counters).  Arguments
// checked by the callers except the ones all share.
static hps_status run_condense(hps_plan *P, hps_prec prec, const double *d_coef, const double *d_f, int m,
                               double tol, int kmax, double *d_S, double *d_T, double *d_h, double *d_W,
                               int *d_info, const double *d_ub, double *d_u, hps_stream stream,
                               const CondenseChunk *ck = nullptr) {
    if (prec != HPS_FP64 && (kmax < 0 || !(tol >= 0.0)))
        return P->fail(HPS_ERR_ARG, "hps_condense: kmax < 0 or tol < 0");
    const bool mixed = prec != HPS_FP64;
    if (mixed && 4 * (P->pmax - 2) + m > 256)
        return P->fail(HPS_ERR_ARG, "hps_condense: mixed precision needs 4(p-2) + m <= 256");
    const size_t tsize = mixed ? sizeof(float) : sizeof(double);
    const int qmax = P->pmax - 2, nmax = qmax * qmax;
    LuBlocking blk = choose_blocking(prec, nmax, P->pmax);
    const int forced = P->forced_nb[mixed ? 1 : 0];
    if (forced) {
        blk.nb_panel = forced;
        if (mixed && (size_t)forced * (blk.ldp + 64) * sizeof(float) <
                         (size_t)(2 * P->pmax * P->pmax + 4 * nmax) * 8)
            return P->fail(HPS_ERR_ARG, "hps_condense: forced panel width too narrow for the refinement staging");
        if (condense_smem(prec, blk) > 227 * 1024)
            return P->fail(HPS_ERR_ARG, "hps_condense: forced panel width needs more than 227 KB of shared memory");
    }
    const int per_sm = condense_max_ctas_per_sm(prec, blk);
    if (per_sm < 1) return P->fail(forced ? HPS_ERR_ARG : HPS_ERR_CUDA, "hps_condense: kernel does not fit on an SM");
    const int full_grid = std::min(P->n_leaves, P->sms * per_sm);
    const int grid = ck ? std::min(ck->n, full_grid) : full_grid;
    long long slot = 0;
    for (int p = P->pmin; p <= P->pmax; ++p) {
        const long long q = p - 2, n = q * q, r = 4 * q + m, C = round_up(n, 4) + r, LDC = round_up(C, 4);
        long long b = n * LDC * (long long)tsize;
        if (mixed) {
            b = round_up(b, 256) + n * r * 8 + 3 * (n + 64) * 4 + 2 * round_up(r, 64) * 4 + n * 12 * 4;   // X, perms, eta, |R_0|, node factors
            b = std::max(b, n * LDC * 8);   // room for the FP64 fallback elimination
        }
        slot = std::max(slot, round_up(b, 256));
    }
    cudaError_t e = P->work.ensure((size_t)slot * full_grid * (ck ? 2 : 1));
    if (e != cudaSuccess) return P->cuda_fail(e, "hps_condense: workspace");
    CondenseParams prm{};
    prm.blk = blk;
    prm.lt = P->leaf_tables();
    prm.dt.dmat = P->d_dmat;
    prm.dt.dmat32 = P->d_dmat32;
    prm.dt.dmat_lo = P->d_dmat_lo;
    prm.dt.doff = P->d_doff;
    prm.n_leaves = P->n_leaves;
    prm.m = m;
    prm.kappa2 = P->kappa * P->kappa;
    prm.coef = d_coef;
    prm.f = m > 0 ? d_f : nullptr;
    prm.S = d_S;
    prm.T = d_T;
    prm.h = m > 0 ? d_h : nullptr;
    prm.W = m > 0 ? d_W : nullptr;
    prm.info = d_info;
    prm.work = (unsigned char *)P->work.p + (ck ? (size_t)ck->half * slot * full_grid : 0);
    prm.slot_bytes = slot;
    prm.queue = P->d_queue;
    if (ck) {
        prm.lt.order = ck->order;
        prm.n_leaves = ck->n;
        prm.queue = ck->queue;
    }
    prm.tol = tol;
    prm.kmax = kmax;
    prm.fallbacks = P->d_queue + 1;
    prm.fallback = P->fallback;
    prm.residual_stop = P->residual_stop;
    prm.ub = d_ub;
    prm.u = d_u;
    cudaStream_t s = (cudaStream_t)stream;
    if (ck) {
        e = launch_condense(prec, prm, grid, s);
        if (e != cudaSuccess) return P->cuda_fail(e, "hps_condense_host: launch");
        return HPS_OK;
    }
    e = cudaMemsetAsync(P->d_queue, 0, 2 * sizeof(int), s);
    P->last_stream = s;
    if (e != cudaSuccess) return P->cuda_fail(e, "hps_condense: queue reset");
    cudaEvent_t *evp = nullptr;
    if (P->timing && P->n_timed < kMaxTimed) {
        evp = P->event_pair(P->n_timed);
        if (evp == nullptr) return P->fail(HPS_ERR_CUDA, "hps_condense: cudaEventCreate failed");
        cudaEventRecord(evp[0], s);
    }
    e = launch_condense(prec, prm, grid, s);
    if (e != cudaSuccess) return P->cuda_fail(e, "hps_condense: launch");
    if (evp) {
        cudaEventRecord(evp[1], s);
        ++P->n_timed;
    }
    P->launches = 1;
    return HPS_OK;
}

hps_status hps_condense(hps_plan *P, hps_prec prec, const double *d_coef, const double *d_f, int m,
                        double tol, int kmax, double *d_S, double *d_T, double *d_h, double *d_W,
                        int *d_info, hps_stream stream) {
    if (P == nullptr) return HPS_ERR_ARG;
    if (prec != HPS_FP64 && prec != HPS_MIXED_FP32 && prec != HPS_MIXED_TF32 && prec != HPS_MIXED_BF16)
        return P->fail(HPS_ERR_ARG, "hps_condense: unknown precision");
    if (d_coef == nullptr || d_T == nullptr || d_info == nullptr)
        return P->fail(HPS_ERR_ARG, "hps_condense: d_coef, d_T and d_info are required");
    if (m < 0) return P->fail(HPS_ERR_ARG, "hps_condense: m < 0");
    if (m > 0 && (d_f == nullptr || d_h == nullptr))
        return P->fail(HPS_ERR_ARG, "hps_condense: m > 0 needs d_f and d_h");
    return run_condense(P, prec, d_coef, d_f, m, tol, kmax, d_S, d_T, d_h, d_W, d_info, nullptr, nullptr, stream);
}

hps_status hps_condense_host(hps_plan *P, hps_prec prec, const double *h_coef, const double *h_f, int m,
                             double tol, int kmax, double *h_S, double *h_T, double *h_h, double *h_W,
                             int *h_info, int chunks, hps_stream stream) {
    if (P == nullptr) return HPS_ERR_ARG;
    if (prec != HPS_FP64 && prec != HPS_MIXED_FP32 && prec != HPS_MIXED_TF32 && prec != HPS_MIXED_BF16)
        return P->fail(HPS_ERR_ARG, "hps_condense_host: unknown precision");
    if (h_coef == nullptr || h_T == nullptr || h_info == nullptr)
        return P->fail(HPS_ERR_ARG, "hps_condense_host: h_coef, h_T and h_info are required");
    if (m < 0) return P->fail(HPS_ERR_ARG, "hps_condense_host: m < 0");
    if (m > 0 && (h_f == nullptr || h_h == nullptr))
        return P->fail(HPS_ERR_ARG, "hps_condense_host: m > 0 needs h_f and h_h");
    if (chunks < 0 || chunks > HPS_HOST_MAX_CHUNKS)
        return P->fail(HPS_ERR_ARG, "hps_condense_host: chunks outside 0..HPS_HOST_MAX_CHUNKS");
    const int nl = P->n_leaves;
    int nc = chunks == 0 ? 8 : chunks;
    nc = std::max(1, std::min(nc, nl));
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    // streams and events, made once per plan
    for (cudaStream_t *sp : {&P->hs_comp, &P->hs_h2d, &P->hs_d2h})
        if (*sp == nullptr && (e = cudaStreamCreateWithFlags(sp, cudaStreamNonBlocking)) != cudaSuccess)
            return P->cuda_fail(e, "hps_condense_host: stream");
    const size_t nev = 3 * (size_t)HPS_HOST_MAX_CHUNKS + 1;
    while (P->hev.size() < nev) {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return P->cuda_fail(e, "hps_condense_host: event");
        P->hev.push_back(ev);
    }
    cudaEvent_t ev_start = P->hev[0];
    auto ev_in = [&](int c) { return P->hev[1 + 3 * c]; };
    auto ev_out = [&](int c) { return P->hev[2 + 3 * c]; };
    auto ev_back = [&](int c) { return P->hev[3 + 3 * c]; };
    // device copies of every input and output, packed as the caller's arrays
    // offsets of leaf l in each packed array for l = 0..nl (the plan keeps
    // the exclusive prefix sums of the first nl leaves)
    auto at = [&](const std::vector<long long> &v, int l, int kind) -> long long {
        if (l < nl) return v[l];
        const long long q = P->p[nl - 1] - 2, sz[5] = {(q + 2) * (q + 2), q * q, 4 * q, q * q * 4 * q, 16 * q * q};
        return v[nl - 1] + sz[kind];
    };
    auto o_p2 = [&](int l) { return at(P->o_p2, l, 0); };
    auto o_ni = [&](int l) { return at(P->o_ni, l, 1); };
    auto o_nb = [&](int l) { return at(P->o_nb, l, 2); };
    auto o_sb = [&](int l) { return at(P->o_sb, l, 3); };
    auto o_bb = [&](int l) { return at(P->o_bb, l, 4); };
    const long long np2 = o_p2(nl), nni = o_ni(nl), nnb = o_nb(nl), nsb = o_sb(nl), nbb = o_bb(nl);
    const size_t b_coef = (size_t)6 * np2 * 8, b_f = (size_t)np2 * m * 8, b_S = h_S ? (size_t)nsb * 8 : 0;
    const size_t b_T = (size_t)nbb * 8, b_h = (size_t)nnb * m * 8, b_W = h_W ? (size_t)nni * m * 8 : 0;
    const size_t o_f = round_up(b_coef, 256), o_S = o_f + round_up(b_f, 256), o_T = o_S + round_up(b_S, 256);
    const size_t o_h = o_T + round_up(b_T, 256), o_W = o_h + round_up(b_h, 256), o_i = o_W + round_up(b_W, 256);
    const size_t o_q = o_i + round_up((size_t)nl * sizeof(int), 256);
    const size_t total = o_q + (size_t)HPS_HOST_MAX_CHUNKS * sizeof(int);
    if ((e = P->hstage.ensure(total)) != cudaSuccess) return P->cuda_fail(e, "hps_condense_host: staging buffers");
    if ((e = P->horder.ensure((size_t)nl * sizeof(int))) != cudaSuccess)
        return P->cuda_fail(e, "hps_condense_host: chunk orders");
    unsigned char *base = (unsigned char *)P->hstage.p;
    double *d_coef = (double *)base, *d_f = m > 0 ? (double *)(base + o_f) : nullptr;
    double *d_S = h_S ? (double *)(base + o_S) : nullptr, *d_T = (double *)(base + o_T);
    double *d_h = m > 0 ? (double *)(base + o_h) : nullptr;
    double *d_W = (h_W && m > 0) ? (double *)(base + o_W) : nullptr;
    int *d_info = (int *)(base + o_i), *d_q = (int *)(base + o_q);
    // contiguous leaf ranges of about equal work (n_i^3), each queued
    // largest leaves first
    std::vector<int> cut(nc + 1, nl);
    {
        std::vector<double> acc(nl + 1, 0.0);
        for (int l = 0; l < nl; ++l) {
            const double ni = (double)(P->p[l] - 2) * (P->p[l] - 2);
            acc[l + 1] = acc[l] + ni * ni * ni;
        }
        cut[0] = 0;
        int l = 0;
        for (int c = 1; c < nc; ++c) {
            const double target = acc[nl] * c / nc;
            while (l < nl && acc[l + 1] <= target) ++l;
            cut[c] = std::max(cut[c - 1] + 1, std::min(l, nl - (nc - c)));
        }
    }
    // the previous call's upload of the orders must be done before the host
    // vector is rewritten
    if ((e = cudaStreamSynchronize(P->hs_h2d)) != cudaSuccess) return P->cuda_fail(e, "hps_condense_host: sync");
    P->horder_host.resize(nl);
    for (int c = 0; c < nc; ++c) {
        int *o = P->horder_host.data() + cut[c];
        for (int l = cut[c]; l < cut[c + 1]; ++l) o[l - cut[c]] = l;
        std::stable_sort(o, o + (cut[c + 1] - cut[c]), [&](int x, int y) { return P->p[x] > P->p[y]; });
    }
    // everything earlier on the caller's stream comes first
    e = cudaMemsetAsync(d_q, 0, (size_t)HPS_HOST_MAX_CHUNKS * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_queue, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaEventRecord(ev_start, s);
    for (cudaStream_t t : {P->hs_comp, P->hs_h2d, P->hs_d2h})
        if (e == cudaSuccess) e = cudaStreamWaitEvent(t, ev_start, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->horder.p, P->horder_host.data(), (size_t)nl * sizeof(int), cudaMemcpyHostToDevice,
                            P->hs_h2d);
    if (e != cudaSuccess) return P->cuda_fail(e, "hps_condense_host: set-up");
    P->last_stream = s;
    auto h2d = [&](void *d, const void *h, size_t off, size_t bytes) {
        return bytes ? cudaMemcpyAsync((char *)d + off, (const char *)h + off, bytes, cudaMemcpyHostToDevice, P->hs_h2d)
                     : cudaSuccess;
    };
    auto d2h = [&](void *h, const void *d, size_t off, size_t bytes) {
        return bytes ? cudaMemcpyAsync((char *)h + off, (const char *)d + off, bytes, cudaMemcpyDeviceToHost, P->hs_d2h)
                     : cudaSuccess;
    };
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
        const int a = cut[c], b = cut[c + 1];
        e = h2d(d_coef, h_coef, (size_t)6 * o_p2(a) * 8, (size_t)6 * (o_p2(b) - o_p2(a)) * 8);
        if (e == cudaSuccess && m > 0)
            e = h2d(d_f, h_f, (size_t)o_p2(a) * m * 8, (size_t)(o_p2(b) - o_p2(a)) * m * 8);
        if (e == cudaSuccess) e = cudaEventRecord(ev_in(c), P->hs_h2d);
        // chunks alternate between the caller's stream and the second compute
        // stream, each with its own half of the workspace
        cudaStream_t cs = (c & 1) ? P->hs_comp : s;
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_in(c), 0);
        if (e != cudaSuccess) break;
        CondenseChunk ck{(const int *)P->horder.p + a, b - a, d_q + c, c & 1};
        hps_status st = run_condense(P, prec, d_coef, d_f, m, tol, kmax, d_S, d_T, d_h, d_W, d_info, nullptr, nullptr,
                                     (hps_stream)cs, &ck);
        if (st != HPS_OK) return st;
        e = cudaEventRecord(ev_out(c), cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(P->hs_d2h, ev_out(c), 0);
        if (e == cudaSuccess && h_S) e = d2h(h_S, d_S, (size_t)o_sb(a) * 8, (size_t)(o_sb(b) - o_sb(a)) * 8);
        if (e == cudaSuccess) e = d2h(h_T, d_T, (size_t)o_bb(a) * 8, (size_t)(o_bb(b) - o_bb(a)) * 8);
        if (e == cudaSuccess && m > 0)
            e = d2h(h_h, d_h, (size_t)o_nb(a) * m * 8, (size_t)(o_nb(b) - o_nb(a)) * m * 8);
        if (e == cudaSuccess && h_W && m > 0)
            e = d2h(h_W, d_W, (size_t)o_ni(a) * m * 8, (size_t)(o_ni(b) - o_ni(a)) * m * 8);
        if (e == cudaSuccess) e = d2h(h_info, d_info, (size_t)a * sizeof(int), (size_t)(b - a) * sizeof(int));
        if (e == cudaSuccess) e = cudaEventRecord(ev_back(c), P->hs_d2h);
    }
    // the call completes on the caller's stream
    // (the copy stream waited for every chunk's launch before its copies)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_back(nc - 1), 0);
    if (e != cudaSuccess) return P->cuda_fail(e, "hps_condense_host");
    P->launches = nc;
    return HPS_OK;
}

hps_status hps_iti_condense(hps_plan *P, double eta, const double *d_coef, const double *d_f, int m, double *d_R,
                            double *d_h, double *d_Y, double *d_uf, int *d_info, hps_stream stream) {
    if (P == nullptr) return HPS_ERR_ARG;
    if (!(eta > 0.0) || !std::isfinite(eta)) return P->fail(HPS_ERR_ARG, "hps_iti_condense: eta must be positive");
    if (m < 0 || d_coef == nullptr || d_R == nullptr || d_info == nullptr || (m > 0 && (d_f == nullptr || d_h == nullptr)))
        return P->fail(HPS_ERR_ARG, "hps_iti_condense: d_coef, d_R, d_info (and d_f, d_h when m > 0) are required");
    const int qmax = P->pmax - 2;
    const LuBlocking blk = iti_blocking(2 * (qmax * qmax + 4 * qmax));
    const int per_sm = iti_max_ctas_per_sm(blk);
    if (per_sm < 1) return P->fail(HPS_ERR_CUDA, "hps_iti_condense: kernel does not fit on an SM");
    const int grid = std::min(P->n_leaves, P->sms * per_sm);
    long long slot = 0;
    for (int p = P->pmin; p <= P->pmax; ++p) {
        const long long q = p - 2, N = q * q + 4 * q, n4 = round_up(2 * N, 4), LDC = round_up(n4 + 4 * q + m, 4);
        slot = std::max(slot, round_up(2 * N * LDC * 8, 256));
    }
    cudaError_t e = P->work.ensure((size_t)slot * grid);
    if (e != cudaSuccess) return P->cuda_fail(e, "hps_iti_condense: workspace");
    CondenseParams prm{};
    prm.blk = blk;
    prm.lt = P->leaf_tables();
    prm.dt.dmat = P->d_dmat;
    prm.dt.dmat32 = P->d_dmat32;
    prm.dt.dmat_lo = P->d_dmat_lo;
    prm.dt.doff = P->d_doff;
    prm.n_leaves = P->n_leaves;
    prm.m = m;
    prm.kappa2 = P->kappa * P->kappa;
    prm.coef = d_coef;
    prm.f = m > 0 ? d_f : nullptr;
    prm.S = d_Y;
    prm.T = d_R;
    prm.h = m > 0 ? d_h : nullptr;
    prm.W = m > 0 ? d_uf : nullptr;
    prm.info = d_info;
    prm.work = (unsigned char *)P->work.p;
    prm.slot_bytes = slot;
    prm.queue = P->d_queue;
    prm.eta = eta;
    cudaStream_t s = (cudaStream_t)stream;
    if ((e = cudaMemsetAsync(P->d_queue, 0, sizeof(int), s)) != cudaSuccess) return P->cuda_fail(e, "hps_iti_condense");
    if ((e = launch_iti(prm, grid, s)) != cudaSuccess) return P->cuda_fail(e, "hps_iti_condense: launch");
    P->launches = 1;
    return HPS_OK;
}

hps_status hps_leaf_resolve(hps_plan *P, hps_prec prec, const double *d_coef, const double *d_f, int m,
                            const double *d_ub, double tol, int kmax, double *d_u, int *d_info,
                            hps_stream stream) {
    if (P == nullptr) return HPS_ERR_ARG;
    if (prec != HPS_FP64 && prec != HPS_MIXED_FP32 && prec != HPS_MIXED_TF32 && prec != HPS_MIXED_BF16)
        return P->fail(HPS_ERR_ARG, "hps_leaf_resolve: unknown precision");
    if (d_coef == nullptr || d_ub == nullptr || d_u == nullptr || d_info == nullptr)
        return P->fail(HPS_ERR_ARG, "hps_leaf_resolve: d_coef, d_ub, d_u and d_info are required");
    if (m < 1) return P->fail(HPS_ERR_ARG, "hps_leaf_resolve: m < 1");
    if (prec != HPS_FP64) prec = HPS_MIXED_FP32;   // m columns only: the FP32 path
    return run_condense(P, prec, d_coef, d_f, m, tol, kmax, nullptr, nullptr, nullptr, nullptr, d_info, d_ub, d_u,
                        stream);
}

hps_status hps_leaf_recover(hps_plan *P, const double *d_S, const double *d_W, int m, const double *d_ub,
                            double *d_u, hps_stream stream) {
    if (P == nullptr) return HPS_ERR_ARG;
    if (d_S == nullptr || d_ub == nullptr || d_u == nullptr)
        return P->fail(HPS_ERR_ARG, "hps_leaf_recover: d_S, d_ub and d_u are required");
    if (m < 1) return P->fail(HPS_ERR_ARG, "hps_leaf_recover: m < 1");
    cudaStream_t s = (cudaStream_t)stream;
    P->last_stream = s;
    cudaError_t e = launch_leaf_recover_all(P->leaf_tables(), P->n_leaves, m, d_S, d_W, d_ub, d_u, s);
    if (e != cudaSuccess) return P->cuda_fail(e, "hps_leaf_recover: launch");
    P->launches = 1;
    return HPS_OK;
}

hps_status hps_set_fp64_fallback(hps_plan *P, int enable) {
    if (P == nullptr) return HPS_ERR_ARG;
    P->fallback = enable != 0;
    return HPS_OK;
}

hps_status hps_set_refine_stop(hps_plan *P, int residual) {
    if (P == nullptr || residual < 0 || residual > 1) return HPS_ERR_ARG;
    P->residual_stop = residual;
    return HPS_OK;
}

hps_status hps_check_info(hps_plan *P, const int *d_info, int n, int *first) {
    auto fail = [&](hps_status st, const std::string &msg) {
        if (P) return P->fail(st, msg);
        g_build_error = msg;
        return st;
    };
    if (first) *first = -1;
    if (n < 0 || (n > 0 && d_info == nullptr)) return fail(HPS_ERR_ARG, "hps_check_info: n >= 0 and d_info required");
    if (n == 0) return HPS_OK;
    std::vector<int> info((size_t)n);
    cudaError_t e = cudaMemcpy(info.data(), d_info, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(HPS_ERR_CUDA, std::string("hps_check_info: ") + cudaGetErrorString(e));
    int pos = -1, neg = -1;
    for (int i = 0; i < n && pos < 0; ++i) {
        if (info[i] > 0) pos = i;
        else if (info[i] < 0 && neg < 0) neg = i;
    }
    if (pos >= 0) {
        if (first) *first = pos;
        return fail(HPS_ERR_SINGULAR, "hps_check_info: entry " + std::to_string(pos) + " has an exact zero pivot at step " +
                                          std::to_string(info[pos]));
    }
    if (neg >= 0) {
        if (first) *first = neg;
        return fail(HPS_ERR_NOCONV, "hps_check_info: entry " + std::to_string(neg) + " did not converge in " +
                                        std::to_string(-info[neg]) + " corrections");
    }
    return HPS_OK;
}

hps_status hps_fallback_count(hps_plan *P, int *count) {
    if (P == nullptr || count == nullptr) return HPS_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(count, P->d_queue + 1, sizeof(int), cudaMemcpyDeviceToHost, P->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->last_stream);
    if (e != cudaSuccess) return P->cuda_fail(e, "hps_fallback_count");
    return HPS_OK;
}

hps_status hps_set_blocking(hps_plan *P, hps_prec prec, int nb_panel) {
    if (P == nullptr) return HPS_ERR_ARG;
    if (prec == HPS_FP64) {
        if (nb_panel != 0 && nb_panel != 4 && nb_panel != 8 && nb_panel != 16)
            return P->fail(HPS_ERR_ARG, "hps_set_blocking: FP64 panel width must be 0, 4, 8 or 16");
        P->forced_nb[0] = nb_panel;
    } else if (prec == HPS_MIXED_FP32 || prec == HPS_MIXED_TF32 || prec == HPS_MIXED_BF16) {
        if (nb_panel != 0 && nb_panel != 8 && nb_panel != 16 && nb_panel != 32)
            return P->fail(HPS_ERR_ARG, "hps_set_blocking: FP32 panel width must be 0, 8, 16 or 32");
        P->forced_nb[1] = nb_panel;
    } else {
        return P->fail(HPS_ERR_ARG, "hps_set_blocking: precision not supported");
    }
    return HPS_OK;
}

hps_status hps_set_timing(hps_plan *P, int enable) {
    if (P == nullptr) return HPS_ERR_ARG;
    P->timing = enable != 0;
    P->n_timed = 0;
    return HPS_OK;
}

hps_status hps_phase_times(hps_plan *P, float *ms, int n) {
    if (P == nullptr || ms == nullptr || n < 1) return HPS_ERR_ARG;
    if (!P->timing || P->n_timed == 0)
        return P->fail(HPS_ERR_STATE, "hps_phase_times: timing not enabled or no call recorded");
    double total = 0.0;
    float last = 0.0f;
    for (int i = 0; i < P->n_timed; ++i) {
        cudaError_t e = cudaEventSynchronize(P->ev[2 * i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&last, P->ev[2 * i], P->ev[2 * i + 1]);
        if (e != cudaSuccess) return P->cuda_fail(e, "hps_phase_times");
        total += last;
    }
    const float vals[3] = {(float)total, (float)P->n_timed, last};
    for (int i = 0; i < n; ++i) ms[i] = i < 3 ? vals[i] : 0.0f;
    return HPS_OK;
}

int hps_last_launch_count(const hps_plan *P) { return P ? P->launches : 0; }

// ---------------------------------------------------------------------------
// Merge tree
// ---------------------------------------------------------------------------

namespace {

struct HostLevel {
    int dir;  // 0: x, 1: y
    int wx, wy;   // child box size in leaves
    int nm, n3, np, nbc;
    std::vector<int> ca, cb, par_child, par_idx, s3a, s3b, srca, srcb;
};

// Boundary of a box of wx x wy leaves: [W (wy q), E (wy q), S (wx q), N (wx q)].
void build_level(int q, int dir, int wx, int wy, int nbx, int nby, HostLevel &H) {
    H.dir = dir;
    H.wx = wx;
    H.wy = wy;
    const int Wc = 0, Ec = wy * q, Sc = 2 * wy * q, Nc = 2 * wy * q + wx * q;
    H.nbc = 2 * (wx + wy) * q;
    if (dir == 0) {
        H.n3 = wy * q;
        H.np = 2 * (2 * wx + wy) * q;
        auto add = [&](int ch, int idx) { H.par_child.push_back(ch); H.par_idx.push_back(idx); };
        for (int k = 0; k < wy * q; ++k) add(0, Wc + k);          // W' = alpha.W
        for (int k = 0; k < wy * q; ++k) add(1, Ec + k);          // E' = beta.E
        for (int k = 0; k < wx * q; ++k) add(0, Sc + k);          // S' = alpha.S, beta.S
        for (int k = 0; k < wx * q; ++k) add(1, Sc + k);
        for (int k = 0; k < wx * q; ++k) add(0, Nc + k);          // N' = alpha.N, beta.N
        for (int k = 0; k < wx * q; ++k) add(1, Nc + k);
        for (int k = 0; k < H.n3; ++k) { H.s3a.push_back(Ec + k); H.s3b.push_back(Wc + k); }
        H.nm = (nbx / 2) * nby;
        for (int px = 0; px < nbx / 2; ++px)
            for (int py = 0; py < nby; ++py) {
                H.ca.push_back((2 * px) * nby + py);
                H.cb.push_back((2 * px + 1) * nby + py);
            }
    } else {
        H.n3 = wx * q;
        H.np = 2 * (wx + 2 * wy) * q;
        auto add = [&](int ch, int idx) { H.par_child.push_back(ch); H.par_idx.push_back(idx); };
        for (int k = 0; k < wy * q; ++k) add(0, Wc + k);          // W' = alpha.W, beta.W
        for (int k = 0; k < wy * q; ++k) add(1, Wc + k);
        for (int k = 0; k < wy * q; ++k) add(0, Ec + k);          // E' = alpha.E, beta.E
        for (int k = 0; k < wy * q; ++k) add(1, Ec + k);
        for (int k = 0; k < wx * q; ++k) add(0, Sc + k);          // S' = alpha.S
        for (int k = 0; k < wx * q; ++k) add(1, Nc + k);          // N' = beta.N
        for (int k = 0; k < H.n3; ++k) { H.s3a.push_back(Nc + k); H.s3b.push_back(Sc + k); }
        H.nm = nbx * (nby / 2);
        for (int px = 0; px < nbx; ++px)
            for (int py = 0; py < nby / 2; ++py) {
                H.ca.push_back(px * nby + 2 * py);
                H.cb.push_back(px * nby + 2 * py + 1);
            }
    }
    H.srca.assign(H.nbc, 0);
    H.srcb.assign(H.nbc, 0);
    for (int k = 0; k < H.n3; ++k) {
        H.srca[H.s3a[k]] = -(k + 1);
        H.srcb[H.s3b[k]] = -(k + 1);
    }
    for (int P = 0; P < H.np; ++P) (H.par_child[P] == 0 ? H.srca : H.srcb)[H.par_idx[P]] = P;
}

bool pow2(int v) { return v >= 1 && (v & (v - 1)) == 0; }

}  // namespace

// The merge tree over an nx x ny grid of unit boxes of wx0 x wy0 leaves
// each (1 x 1: the leaves of hps_condense), whose DtN maps and fluxes are
// d_T, d_h; with d_root_Th the root's own [T | h] is formed there too.
static hps_status merge_tree(hps_plan *P, const char *who, int nx, int ny, int wx0, int wy0, const double *d_T,
                             const double *d_h, int m, double *d_root_Th, hps_stream stream, int tx = 0, int ty = 0) {
    if (P == nullptr) return HPS_ERR_ARG;
    if (!P->uniform) return P->fail(HPS_ERR_ARG, std::string(who) + ": needs one p on every leaf");
    if (!pow2(nx) || !pow2(ny) || !pow2(wx0) || !pow2(wy0) || (long long)nx * ny != P->n_leaves)
        return P->fail(HPS_ERR_ARG, std::string(who) + ": nx, ny, wx0, wy0 must be powers of two with nx*ny = n_leaves");
    if (d_T == nullptr || m < 0 || (m > 0 && d_h == nullptr))
        return P->fail(HPS_ERR_ARG, std::string(who) + ": d_T required, d_h required when m > 0");
    const int q = P->pmin - 2;
    cudaStream_t s = (cudaStream_t)stream;
    P->merged = false;
    P->slabbed = false;
    const int split_below = P->split_below < 0 ? P->sms : P->split_below;
    const int NX = nx * wx0, NY = ny * wy0;   // the whole grid, in leaves
    // merges stop at boxes of tx x ty leaves (default: the whole grid; the
    // slabs of SlabLU stop at s x NY): x merges while below tx, alternating
    // with y as in the full tree
    if (tx <= 0) tx = NX;
    if (ty <= 0) ty = NY;
    int wx = wx0, wy = wy0;
    std::vector<HostLevel> hl;
    while (wx < tx || wy < ty) {
        const int dir = (wx < tx && (wx <= wy || wy == ty)) ? 0 : 1;
        HostLevel H;
        build_level(q, dir, wx, wy, NX / wx, NY / wy, H);
        hl.push_back(H);
        if (dir == 0) wx *= 2; else wy *= 2;
    }
    // the level buffers of an earlier call are kept (ensure() grows them);
    // levels beyond this tree's depth are freed
    for (size_t i = hl.size(); i < P->levels.size(); ++i) {
        Level &L = P->levels[i];
        L.maps.release(); L.aug.release(); L.th.release(); L.u.release(); L.info.release();
        L.piv.release(); L.u3.release(); L.oz.release();
    }
    P->levels.resize(hl.size());
    cudaError_t e = cudaSuccess;
    const int nbc0 = 2 * (wx0 + wy0) * q;   // boundary nodes of a unit box
    bool used_oz = false;
    if (P->merge_tensor) {
        if ((e = P->oz_err.ensure(sizeof(int))) != cudaSuccess) return P->cuda_fail(e, who);
        if ((e = cudaMemsetAsync(P->oz_err.p, 0, sizeof(int), s)) != cudaSuccess) return P->cuda_fail(e, who);
    }
    if (hl.empty() && d_root_Th) {
        // one unit box: the root is the box itself
        e = cudaMemcpy2DAsync(d_root_Th, (size_t)(nbc0 + m) * sizeof(double), d_T, (size_t)nbc0 * sizeof(double),
                              (size_t)nbc0 * sizeof(double), nbc0, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && m > 0)
            e = cudaMemcpy2DAsync(d_root_Th + nbc0, (size_t)(nbc0 + m) * sizeof(double), d_h, (size_t)m * sizeof(double),
                                  (size_t)m * sizeof(double), nbc0, cudaMemcpyDeviceToDevice, s);
    }
    // every level's index maps reach the device before the first launch, so
    // the copies (from pageable memory, which wait for the stream) do not
    // hold the host back between the levels' kernels
    std::vector<std::vector<int>> all_maps(hl.size());
    std::vector<std::array<size_t, 8>> offs(hl.size());
    for (size_t li = 0; li < hl.size() && e == cudaSuccess; ++li) {
        const HostLevel &H = hl[li];
        std::vector<int> &maps = all_maps[li];
        auto put = [&](const std::vector<int> &v) { size_t o = maps.size(); maps.insert(maps.end(), v.begin(), v.end()); return o; };
        offs[li] = {put(H.ca), put(H.cb), put(H.par_child), put(H.par_idx), put(H.s3a), put(H.s3b), put(H.srca),
                    put(H.srcb)};
        if ((e = P->levels[li].maps.ensure(maps.size() * sizeof(int))) != cudaSuccess) break;
        e = cudaMemcpyAsync(P->levels[li].maps.p, maps.data(), maps.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (size_t li = 0; li < hl.size() && e == cudaSuccess; ++li) {
        const HostLevel &H = hl[li];
        Level &L = P->levels[li];
        const size_t oca = offs[li][0], ocb = offs[li][1], opc = offs[li][2], opi = offs[li][3];
        const size_t o3a = offs[li][4], o3b = offs[li][5], osa = offs[li][6], osb = offs[li][7];
        const bool root = li + 1 == hl.size();
        const bool form = !root || d_root_Th != nullptr;
        const int lda = (int)round_up(round_up(H.n3, 4) + H.np + m, 4);
        if ((e = L.aug.ensure((size_t)H.nm * H.n3 * lda * sizeof(double))) != cudaSuccess) break;
        if (!root && (e = L.th.ensure((size_t)H.nm * H.np * (H.np + m) * sizeof(double))) != cudaSuccess) break;
        if ((e = L.u.ensure((size_t)H.nm * H.np * std::max(m, 1) * sizeof(double))) != cudaSuccess) break;
        if ((e = L.info.ensure((size_t)H.nm * sizeof(int))) != cudaSuccess) break;
        if ((e = L.u3.ensure((size_t)H.nm * H.n3 * std::max(m, 1) * sizeof(double))) != cudaSuccess) break;
        const bool split = H.nm < split_below && split_solve_fits(H.n3);
        if (split && (e = L.piv.ensure((size_t)H.nm * H.n3 * sizeof(int))) != cudaSuccess) break;
        const int *mp = (const int *)L.maps.p;
        MergeLevelDev &D = L.dev;
        D.nm = H.nm; D.n3 = H.n3; D.c3 = (int)round_up(H.n3, 4); D.np = H.np; D.nbc = H.nbc; D.m = m; D.lda = lda;
        D.ca = mp + oca; D.cb = mp + ocb; D.par_child = mp + opc; D.par_idx = mp + opi;
        D.s3a = mp + o3a; D.s3b = mp + o3b; D.srca = mp + osa; D.srcb = mp + osb;
        D.leaf_T = li == 0 ? d_T : nullptr;
        D.leaf_h = li == 0 ? (m > 0 ? d_h : nullptr) : nullptr;
        D.prev_Th = li == 0 ? nullptr : (const double *)P->levels[li - 1].th.p;
        D.aug = (double *)L.aug.p;
        D.Th = root ? d_root_Th : (double *)L.th.p;
        D.info = (int *)L.info.p;
        D.ipiv = split ? (int *)L.piv.p : nullptr;
        D.u3 = (double *)L.u3.p;
        if (split && P->split_aux.side == nullptr) {
            if ((e = cudaStreamCreateWithFlags(&P->split_aux.side, cudaStreamNonBlocking)) != cudaSuccess) break;
            if ((e = cudaEventCreateWithFlags(&P->split_aux.a, cudaEventDisableTiming)) != cudaSuccess) break;
            if ((e = cudaEventCreateWithFlags(&P->split_aux.b, cudaEventDisableTiming)) != cudaSuccess) break;
        }
        D.use_oz = form && P->merge_tensor && ozaki_applies(H.np, H.n3);
        D.oz_solve = split && P->merge_tensor && split_solve_blocked(H.n3, H.np + m);
        if (D.use_oz || D.oz_solve) {
            size_t bytes = 0;
            if (D.use_oz) bytes = ozaki_scratch_bytes(H.nm, H.np, H.n3, H.np + m);
            if (D.oz_solve) bytes = std::max(bytes, split_solve_scratch(H.nm, H.n3, H.np + m));
            if ((e = L.oz.ensure(bytes)) != cudaSuccess) break;
            D.oz = ozaki_layout(L.oz.p, H.nm, H.np, H.n3, H.np + m, (int *)P->oz_err.p);
            used_oz = true;
        }
        if ((e = launch_merge_level(D, form, s, split ? &P->split_aux : nullptr)) != cudaSuccess) break;
    }
    if (e == cudaSuccess && used_oz) {   // a tensor-core wait that timed out left its tile unwritten
        int flag = 0;
        e = cudaMemcpyAsync(&flag, P->oz_err.p, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && flag) return P->fail(HPS_ERR_CUDA, std::string(who) + ": a tensor-core wait timed out");
    }
    // an exactly singular Z (zero pivot) leaves inf / NaN in the maps: say where
    for (size_t li = 0; li < hl.size() && e == cudaSuccess; ++li) {
        std::vector<int> info((size_t)hl[li].nm);
        e = cudaMemcpyAsync(info.data(), P->levels[li].info.p, info.size() * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (size_t k = 0; k < info.size() && e == cudaSuccess; ++k)
            if (info[k] > 0)
                return P->fail(HPS_ERR_SINGULAR, std::string(who) + ": level " + std::to_string(li) + ", merge " +
                                                     std::to_string(k) + ": exact zero pivot in Z at step " +
                                                     std::to_string(info[k]));
    }
    if (e != cudaSuccess) return P->cuda_fail(e, who);
    if ((e = P->u_leaf.ensure((size_t)P->n_leaves * nbc0 * std::max(m, 1) * sizeof(double))) != cudaSuccess)
        return P->cuda_fail(e, "merge: unit-box boundary buffer");
    P->merge_nx = nx;
    P->merge_ny = ny;
    P->merge_wx0 = wx0;
    P->merge_wy0 = wy0;
    P->merge_m = m;
    P->merged = true;
    P->launches = 0;
    for (auto &L : P->levels) {
        P->launches += 1 + (L.dev.Th ? (L.dev.use_oz ? 4 : 1) : 0) +
                       (L.dev.ipiv ? split_solve_launches(L.dev.n3, L.dev.np + L.dev.m, L.dev.oz_solve != 0, true) : 1);
    }
    return HPS_OK;
}

hps_status hps_merge(hps_plan *P, int nx, int ny, const double *d_T, const double *d_h, int m,
                     hps_stream stream) {
    return merge_tree(P, "hps_merge", nx, ny, 1, 1, d_T, d_h, m, nullptr, stream);
}

hps_status hps_merge_boxes(hps_plan *P, int nx, int ny, int wx0, int wy0, const double *d_T, const double *d_h, int m,
                           double *d_root_Th, hps_stream stream) {
    return merge_tree(P, "hps_merge_boxes", nx, ny, wx0, wy0, d_T, d_h, m, d_root_Th, stream);
}

hps_status hps_set_merge_tensor(hps_plan *P, int enable) {
    if (P == nullptr || enable < 0 || enable > 2) return HPS_ERR_ARG;
    P->merge_tensor = enable;
    return HPS_OK;
}

hps_status hps_set_merge_split(hps_plan *P, int below) {
    if (P == nullptr || below < -1) return HPS_ERR_ARG;
    P->split_below = below;
    return HPS_OK;
}

// The downward pass through the stored levels: from the top level's parent
// values upar (one block of np x m per merge of that level) to the unit
// boxes' boundary values in dst.
static cudaError_t down_levels(hps_plan *P, const double *upar, double *dst, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    const int nl = (int)P->levels.size();
    for (int li = nl - 1; li >= 0 && e == cudaSuccess; --li) {
        const Level &L = P->levels[li];
        // parents of level li are the children of level li + 1, whose values
        // the previous iteration wrote into L.u; the top level takes upar
        const double *up = (li == nl - 1) ? upar : (const double *)L.u.p;
        double *uch = li > 0 ? (double *)P->levels[li - 1].u.p : dst;
        e = launch_merge_down(L.dev, up, uch, s);
    }
    return e;
}

// Top-down pass of the last merge: the unit boxes' boundary values into
// ub (the plan's buffer when null), n_leaves x nbc0 x m.
static hps_status solve_down(hps_plan *P, const char *who, const double *d_g, int m, double *ub, hps_stream stream,
                             const double **ub_out) {
    if (!P->merged) return P->fail(HPS_ERR_STATE, std::string(who) + ": call hps_merge first");
    if (m < 1 || m != P->merge_m)
        return P->fail(HPS_ERR_ARG, std::string(who) + ": m must equal the m of the merge and be >= 1");
    if (d_g == nullptr) return P->fail(HPS_ERR_ARG, std::string(who) + ": d_g is required");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    const int nl = (int)P->levels.size();
    double *dst = ub ? ub : (double *)P->u_leaf.p;
    if (nl == 0) {
        const int q = P->pmin - 2, nbc0 = 2 * (P->merge_wx0 + P->merge_wy0) * q;
        e = cudaMemcpyAsync(dst, d_g, (size_t)nbc0 * m * sizeof(double), cudaMemcpyDeviceToDevice, s);
    } else {
        e = down_levels(P, d_g, dst, s);
    }
    if (e != cudaSuccess) return P->cuda_fail(e, who);
    *ub_out = dst;
    P->launches = 2 * nl;
    return HPS_OK;
}

hps_status hps_solve(hps_plan *P, const double *d_g, const double *d_S, const double *d_W, int m,
                     double *d_u, hps_stream stream) {
    if (P == nullptr) return HPS_ERR_ARG;
    if (P->merged && (P->merge_wx0 != 1 || P->merge_wy0 != 1))
        return P->fail(HPS_ERR_STATE, "hps_solve: the last merge was over boxes (use hps_solve_boxes)");
    if (d_S == nullptr || d_u == nullptr) return P->fail(HPS_ERR_ARG, "hps_solve: d_g, d_S and d_u are required");
    const double *ub = nullptr;
    const hps_status st = solve_down(P, "hps_solve", d_g, m, nullptr, stream, &ub);
    if (st != HPS_OK) return st;
    const cudaError_t e = launch_leaf_recover(P->n_leaves, P->pmin, m, d_S, d_W, ub, d_u, (cudaStream_t)stream);
    if (e != cudaSuccess) return P->cuda_fail(e, "hps_solve: leaf recovery");
    P->launches += 1;
    return HPS_OK;
}

hps_status hps_solve_boxes(hps_plan *P, const double *d_g, int m, double *d_ub, hps_stream stream) {
    if (P == nullptr) return HPS_ERR_ARG;
    if (d_ub == nullptr) return P->fail(HPS_ERR_ARG, "hps_solve_boxes: d_ub is required");
    const double *ub = nullptr;
    return solve_down(P, "hps_solve_boxes", d_g, m, d_ub, stream, &ub);
}

// ---------------------------------------------------------------------------
// SlabLU (slab.cu): slab merges, block LU of the interface system, solve
// ---------------------------------------------------------------------------

hps_status hps_slab_factor(hps_plan *P, int nx, int ny, int s, const double *d_T, const double *d_h, int m,
                           hps_stream stream) {
    if (P == nullptr) return HPS_ERR_ARG;
    if (!pow2(s) || s < 2 || s > nx)
        return P->fail(HPS_ERR_ARG, "hps_slab_factor: the slab width s must be a power of two, 2 <= s <= nx");
    if (m < 1) return P->fail(HPS_ERR_ARG, "hps_slab_factor: m >= 1 body-load columns are required");
    const int q = P->pmin - 2, n = ny * q, S = nx / s, nps = 2 * (s + ny) * q, ldt = nps + m;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = P->slab_th.ensure((size_t)S * nps * ldt * sizeof(double));
    if (e != cudaSuccess) return P->cuda_fail(e, "hps_slab_factor: slab maps");
    // the slabs' interiors: merges inside every slab up to its [T | h]
    hps_status r = merge_tree(P, "hps_slab_factor", nx, ny, 1, 1, d_T, d_h, m, (double *)P->slab_th.p, stream, s, ny);
    if (r != HPS_OK) return r;
    P->merged = false;   // the stored levels stop at the slabs: only hps_slab_solve uses them
    int launches = P->launches;
    if (S > 1) {
        const int c3 = (int)round_up(n, 4), lda = (int)round_up(c3 + 2 * n + m, 4);
        if ((e = P->slab_aug.ensure((size_t)(S - 1) * n * lda * sizeof(double))) != cudaSuccess ||
            (e = P->slab_piv.ensure((size_t)(S - 1) * n * sizeof(int))) != cudaSuccess ||
            (e = P->slab_info.ensure((size_t)(S - 1) * sizeof(int))) != cudaSuccess)
            return P->cuda_fail(e, "hps_slab_factor: interface systems");
        const bool split = split_solve_fits(n);
        if (split && P->split_aux.side == nullptr) {
            if ((e = cudaStreamCreateWithFlags(&P->split_aux.side, cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&P->split_aux.a, cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&P->split_aux.b, cudaEventDisableTiming)) != cudaSuccess)
                return P->cuda_fail(e, "hps_slab_factor: streams");
        }
        double *aug = (double *)P->slab_aug.p;
        const double *th = (const double *)P->slab_th.p;
        const bool blocked = split && P->merge_tensor == 2 && split_solve_blocked(n, 2 * n + m);
        OzakiScratch oz{};
        if (blocked) {
            if ((e = P->slab_oz.ensure(split_solve_scratch(1, n, 2 * n + m))) != cudaSuccess ||
                (e = P->oz_err.ensure(sizeof(int))) != cudaSuccess ||
                (e = cudaMemsetAsync(P->oz_err.p, 0, sizeof(int), st)) != cudaSuccess)
                return P->cuda_fail(e, "hps_slab_factor: tensor-core scratch");
            oz = ozaki_layout(P->slab_oz.p, 1, n, n, 2 * n + m, (int *)P->oz_err.p);
        }
        for (int k = 0; k < S - 1 && e == cudaSuccess; ++k) {
            SlabStepDev D{};
            D.n = n; D.m = m; D.ldt = ldt; D.np = nps; D.lda = lda; D.c3 = c3; D.last = k == S - 2;
            D.left = th + (size_t)k * nps * ldt;
            D.right = th + (size_t)(k + 1) * nps * ldt;
            D.prev = k > 0 ? aug + (size_t)(k - 1) * n * lda : nullptr;
            D.aug = aug + (size_t)k * n * lda;
            if ((e = launch_slab_assemble(D, st)) != cudaSuccess) break;
            MergeLevelDev L{};
            L.nm = 1; L.n3 = n; L.c3 = c3; L.np = 2 * n; L.nbc = 0; L.m = m; L.lda = lda;
            L.aug = D.aug;
            L.info = (int *)P->slab_info.p + k;
            L.ipiv = (int *)P->slab_piv.p + (size_t)k * n;
            L.oz_solve = blocked;
            L.oz = oz;
            e = split ? launch_split_solve(L, L.ipiv, st, &P->split_aux)
                      : launch_dense_solve(D.aug, 0, n, c3, c3 + 2 * n + m, lda, 1, L.info, st);
            launches += 2 + (split ? split_solve_launches(n, 2 * n + m, blocked, true) : 1);
        }
        if (e == cudaSuccess && blocked) {   // a tensor-core wait that timed out left its tile unwritten
            int flag = 0;
            e = cudaMemcpyAsync(&flag, P->oz_err.p, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess && flag) return P->fail(HPS_ERR_CUDA, "hps_slab_factor: a tensor-core wait timed out");
        }
        if (e != cudaSuccess) return P->cuda_fail(e, "hps_slab_factor: interface block LU");
    }
    if ((e = P->slab_tmp.ensure((size_t)(2 * (S + 1) * n + (size_t)S * nps) * m * sizeof(double))) != cudaSuccess)
        return P->cuda_fail(e, "hps_slab_factor: solve scratch");
    P->slab_nx = nx; P->slab_ny = ny; P->slab_s = s; P->slab_m = m;
    P->slabbed = true;
    P->launches = launches;
    return HPS_OK;
}

hps_status hps_slab_solve(hps_plan *P, const double *d_g, const double *d_S, const double *d_W, int m, double *d_u,
                          hps_stream stream) {
    if (P == nullptr) return HPS_ERR_ARG;
    if (!P->slabbed) return P->fail(HPS_ERR_STATE, "hps_slab_solve: call hps_slab_factor first");
    if (m != P->slab_m) return P->fail(HPS_ERR_ARG, "hps_slab_solve: m must equal the m of hps_slab_factor");
    if (d_g == nullptr || d_S == nullptr || d_u == nullptr)
        return P->fail(HPS_ERR_ARG, "hps_slab_solve: d_g, d_S and d_u are required");
    const int q = P->pmin - 2, nx = P->slab_nx, ny = P->slab_ny, s = P->slab_s;
    const int n = ny * q, S = nx / s, sq = s * q, nxq = nx * q, nps = 2 * (s + ny) * q, ldt = nps + m;
    const int c3 = (int)round_up(n, 4), lda = (int)round_up(c3 + 2 * n + m, 4);
    cudaStream_t st = (cudaStream_t)stream;
    const double *th = (const double *)P->slab_th.p, *aug = (const double *)P->slab_aug.p;
    double *t = (double *)P->slab_tmp.p;                    // n x m
    double *vg = t + (size_t)n * m;                          // (S - 1) blocks n x m
    double *u = vg + (size_t)S * n * m;                      // (S - 1) blocks n x m
    double *ubs = u + (size_t)S * n * m;                     // S blocks nps x m
    const double *gW = d_g, *gE = d_g + (size_t)n * m, *gS = d_g + (size_t)2 * n * m, *gN = gS + (size_t)nxq * m;
    cudaError_t e = cudaSuccess;
    int launches = 0;
    auto gemv = [&](const double *A, long long la, int rows, int cols, const double *x, int ldx, double *y, double alpha,
                    double beta, const double *add, int ldadd) {
        if (e == cudaSuccess) e = launch_gemv(A, la, rows, cols, x, ldx, y, m, m, alpha, beta, add, ldadd, st);
        ++launches;
    };
    // forward: v^g_k = G_k (b^g_k - L_k v^g_{k-1}), b^g_k from the outer data
    for (int k = 0; k < S - 1; ++k) {
        const double *Tk = th + (size_t)k * nps * ldt, *Tk1 = th + (size_t)(k + 1) * nps * ldt;
        const double *TkE = Tk + (size_t)n * ldt;           // slab k, E rows
        gemv(TkE + 2 * n, ldt, n, sq, gS + (size_t)k * sq * m, m, t, -1.0, 0.0, nullptr, 0);
        gemv(TkE + 2 * n + sq, ldt, n, sq, gN + (size_t)k * sq * m, m, t, -1.0, 1.0, nullptr, 0);
        gemv(Tk1 + 2 * n, ldt, n, sq, gS + (size_t)(k + 1) * sq * m, m, t, -1.0, 1.0, nullptr, 0);
        gemv(Tk1 + 2 * n + sq, ldt, n, sq, gN + (size_t)(k + 1) * sq * m, m, t, -1.0, 1.0, nullptr, 0);
        if (k == 0) gemv(TkE, ldt, n, n, gW, m, t, -1.0, 1.0, nullptr, 0);                 // outer W data
        else gemv(TkE, ldt, n, n, vg + (size_t)(k - 1) * n * m, m, t, -1.0, 1.0, nullptr, 0);   // - L_k v^g_{k-1}
        if (k == S - 2) gemv(Tk1 + n, ldt, n, n, gE, m, t, -1.0, 1.0, nullptr, 0);         // outer E data
        gemv(aug + (size_t)k * n * lda + c3 + n, lda, n, n, t, m, vg + (size_t)k * n * m, 1.0, 0.0, nullptr, 0);
    }
    // back: u_k = v^g_k + v^h_k + S_k u_{k+1}
    for (int k = S - 2; k >= 0; --k) {
        const double *ak = aug + (size_t)k * n * lda;
        double *uk = u + (size_t)k * n * m;
        if (k == S - 2) gemv(ak, lda, n, 0, t, m, uk, 0.0, 0.0, vg + (size_t)k * n * m, m);
        else gemv(ak + c3, lda, n, n, u + (size_t)(k + 1) * n * m, m, uk, 1.0, 0.0, vg + (size_t)k * n * m, m);
        gemv(ak, lda, n, 0, t, m, uk, 0.0, 1.0, ak + c3 + 2 * n, lda);
    }
    // every slab's boundary values, the downward pass inside the slabs, the leaves
    if (e == cudaSuccess) e = launch_slab_bounds(S, n, sq, nxq, m, u, d_g, ubs, st);
    if (e == cudaSuccess) e = down_levels(P, ubs, (double *)P->u_leaf.p, st);
    if (e == cudaSuccess) e = launch_leaf_recover(P->n_leaves, P->pmin, m, d_S, d_W, (const double *)P->u_leaf.p, d_u, st);
    if (e != cudaSuccess) return P->cuda_fail(e, "hps_slab_solve");
    P->launches = launches + 2 + 2 * (int)P->levels.size();
    return HPS_OK;
}

void hps_destroy(hps_plan *P) {
    if (P == nullptr) return;
    cudaDeviceSynchronize();
    for (auto &L : P->levels) {
        L.maps.release(); L.aug.release(); L.th.release(); L.u.release(); L.info.release();
        L.piv.release(); L.u3.release(); L.oz.release();
    }
    P->u_leaf.release();
    P->oz_err.release();
    P->slab_oz.release();
    P->slab_th.release(); P->slab_aug.release(); P->slab_piv.release(); P->slab_info.release(); P->slab_tmp.release();
    P->hstage.release();
    P->horder.release();
    for (cudaStream_t t : {P->hs_comp, P->hs_h2d, P->hs_d2h, P->split_aux.side})
        if (t) cudaStreamDestroy(t);
    for (cudaEvent_t ev : {P->split_aux.a, P->split_aux.b})
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : P->hev) cudaEventDestroy(ev);
    P->work.release();
    P->tables.release();
    for (cudaEvent_t ev : P->ev) cudaEventDestroy(ev);
    delete P;
}

}  // extern "C"
