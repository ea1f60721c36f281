// hps_condense_noalloc: FP64 leaf condensation that allocates no device
// memory.  Everything the condensation kernel needs beyond the caller's
// inputs and outputs (the per-leaf tables, the Chebyshev matrices, the work
// counter and the per-CTA elimination workspace) lives in one file-scope
// __device__ array of fixed size, so a call only launches kernels.
//
// Who needs this: callers that cannot call cudaMalloc at the time they
// condense -- for example code running inside a host framework that owns all
// device memory through its own pool and forbids outside allocations (to
// keep a fixed memory budget), or a latency-critical service loop where an
// allocation could block on device synchronisation or fail under memory
// pressure.  They pass inputs and outputs they already own; the plan-based
// hps_build_leaves / hps_condense pair allocates its tables and workspace
// and is not usable there.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "hps.h"
#include "hps_internal.cuh"

namespace hps {
void set_global_error(const std::string &msg);  // hps_api.cu: text of hps_last_error(NULL)
}

namespace {

using namespace hps;

// The scratch array: 32 MiB on every GPU that loads this library, held
// until the process exits.  Shared by all calls on a device; it keeps the
// last call's contents, and everything that must start at zero is cleared
// by each call.
constexpr size_t kScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Device address of the scratch array in the current device's context (host
// code must not use g_scratch itself: on the host it is only a stand-in
// symbol).  Looked up on every call rather than cached: a cached address
// would dangle once cudaDeviceReset or a re-created primary context reloads
// the module.  After the first call on a device (which loads the module)
// the lookup is a host-side table query.
cudaError_t scratch_address(void **out) { return cudaGetSymbolAddress(out, g_scratch); }

// Per-call set-up in the scratch: uniform-p leaf tables (order p, packed
// offsets, identity work order), the Chebyshev matrix D of order p on
// [-1, 1], D*D and the corner extrapolation weights, and a zeroed work
// counter.  D follows the same definition
// as the plan path (barycentric weights, product form of the node
// differences, diagonal from the zero row sum).
__global__ void noalloc_setup(int n_leaves, int p, int *pv, long long *off, int *order, int *doff,
                              double *dmat, int *queue) {
    const long long q = p - 2;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n_leaves; l += gridDim.x * blockDim.x) {
        pv[l] = p;
        off[l] = (long long)l * p * p;
        off[n_leaves + l] = (long long)l * q * q;
        off[2LL * n_leaves + l] = (long long)l * 4 * q;
        off[3LL * n_leaves + l] = (long long)l * q * q * 4 * q;
        off[4LL * n_leaves + l] = (long long)l * 16 * q * q;
        order[l] = l;
    }
    if (blockIdx.x != 0) return;
    for (int t = threadIdx.x; t <= HPS_PMAX; t += blockDim.x) doff[t] = (t == p) ? 0 : -1;
    if (threadIdx.x == 0) *queue = 0;
    const int N = p - 1;
    double *D = dmat, *D2 = dmat + p * p;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        if (i == j) continue;
        const double wi = ((i & 1) ? -1.0 : 1.0) * ((i == 0 || i == N) ? 0.5 : 1.0);
        const double wj = ((j & 1) ? -1.0 : 1.0) * ((j == 0 || j == N) ? 0.5 : 1.0);
        const double diff = 2.0 * sinpi((i + j) / (2.0 * N)) * sinpi((i - j) / (2.0 * N));
        D[e] = (wj / wi) / diff;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < p; ++j)
            if (j != i) s += D[i * p + j];
        D[i * p + i] = -s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        double s = 0.0;
        for (int k = 0; k < p; ++k) s += D[i * p + k] * D[k * p + j];
        D2[e] = s;
    }
    // corner extrapolation weights, as the plan path: the Lagrange basis of
    // the interior nodes t_1..t_q at -1 and +1, halved (barycentric form)
    double *ce = D2 + p * p;
    for (int e = threadIdx.x; e < 2 * p; e += blockDim.x) {
        const int side = e / p, l = e % p;
        double v = 0.0;
        if (l >= 1 && l <= q) {
            const double s = side ? 1.0 : -1.0;
            double den = 0.0, num = 0.0;
            for (int k = 1; k <= q; ++k) {
                const double tk = -cospi((double)k / N);
                double w = 1.0;
                for (int mm = 1; mm <= q; ++mm)
                    if (mm != k) w *= (tk + cospi((double)mm / N));
                const double term = (1.0 / w) / (s - tk);
                den += term;
                if (k == l) num = term;
            }
            v = 0.5 * num / den;
        }
        ce[e] = v;
    }
}

hps_status fail(hps_status s, const std::string &msg) {
    set_global_error("hps_condense_noalloc: " + msg);
    return s;
}

}  // namespace

extern "C" hps_status hps_condense_noalloc(int n_leaves, int p, double kappa, const double *d_box,
                                           const double *d_coef, const double *d_f, int m, double *d_S,
                                           double *d_T, double *d_h, double *d_W, int *d_info,
                                           hps_stream stream) {
    if (n_leaves < 1 || p < HPS_PMIN || p > HPS_PMAX || m < 0 || !std::isfinite(kappa))
        return fail(HPS_ERR_ARG, "n_leaves >= 1, HPS_PMIN <= p <= HPS_PMAX, m >= 0 and a finite kappa are required");
    if (d_box == nullptr || d_coef == nullptr || d_T == nullptr || d_info == nullptr ||
        (m > 0 && (d_f == nullptr || d_h == nullptr)))
        return fail(HPS_ERR_ARG, "d_box, d_coef, d_T, d_info (and d_f, d_h when m > 0) are required");
    // scratch layout: tables, then 256-byte aligned workspace slots
    const size_t nl = (size_t)n_leaves;
    const size_t o_p = 0, o_off = align256(o_p + nl * sizeof(int));
    const size_t o_ord = align256(o_off + 5 * nl * sizeof(long long));
    const size_t o_doff = align256(o_ord + nl * sizeof(int));
    const size_t o_dmat = align256(o_doff + (HPS_PMAX + 1) * sizeof(int));
    const size_t o_queue = align256(o_dmat + (2 * (size_t)p * p + 2 * (size_t)p) * sizeof(double));
    const size_t o_work = align256(o_queue + sizeof(int));
    const long long q = p - 2, n = q * q, r = 4 * q + m, C = ((n + 3) & ~3LL) + r, LDC = (C + 3) & ~3LL;
    const size_t slot = align256((size_t)(n * LDC) * sizeof(double));
    if (o_work + slot > kScratchBytes)
        return fail(HPS_ERR_ARG, "tables plus one leaf workspace need " + std::to_string(o_work + slot) +
                                     " bytes; the scratch holds " + std::to_string(kScratchBytes) +
                                     " (fewer leaves, smaller p or m)");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(HPS_ERR_CUDA, cudaGetErrorString(e));
    void *base_v = nullptr;
    e = scratch_address(&base_v);
    if (e != cudaSuccess) return fail(HPS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    unsigned char *base = (unsigned char *)base_v;
    const LuBlocking blk = choose_blocking(HPS_FP64, (int)n, p);
    const int per_sm = condense_max_ctas_per_sm(HPS_FP64, blk);
    if (per_sm < 1) return fail(HPS_ERR_CUDA, "kernel does not fit on an SM");
    const long long slots = (long long)((kScratchBytes - o_work) / slot);
    const int grid = (int)std::min<long long>({(long long)n_leaves, (long long)sms * per_sm, slots});
    CondenseParams prm{};
    prm.blk = blk;
    prm.lt.p = (const int *)(base + o_p);
    prm.lt.box = d_box;
    const long long *off = (const long long *)(base + o_off);
    prm.lt.o_p2 = off;
    prm.lt.o_ni = off + nl;
    prm.lt.o_nb = off + 2 * nl;
    prm.lt.o_sb = off + 3 * nl;
    prm.lt.o_bb = off + 4 * nl;
    prm.lt.order = (const int *)(base + o_ord);
    prm.dt.dmat = (const double *)(base + o_dmat);
    prm.dt.doff = (const int *)(base + o_doff);
    prm.n_leaves = n_leaves;
    prm.m = m;
    prm.kappa2 = kappa * kappa;
    prm.coef = d_coef;
    prm.f = m > 0 ? d_f : nullptr;
    prm.S = d_S;
    prm.T = d_T;
    prm.h = m > 0 ? d_h : nullptr;
    prm.W = m > 0 ? d_W : nullptr;
    prm.info = d_info;
    prm.work = base + o_work;
    prm.slot_bytes = (long long)slot;
    prm.queue = (int *)(base + o_queue);
    cudaStream_t s = (cudaStream_t)stream;
    const int sg = (int)std::min<size_t>((nl + 255) / 256, 1024);
    noalloc_setup<<<sg, 256, 0, s>>>(n_leaves, p, (int *)(base + o_p), (long long *)(base + o_off),
                                     (int *)(base + o_ord), (int *)(base + o_doff), (double *)(base + o_dmat),
                                     (int *)(base + o_queue));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_condense(HPS_FP64, prm, grid, s);
    if (e != cudaSuccess) return fail(HPS_ERR_CUDA, cudaGetErrorString(e));
    return HPS_OK;
}
