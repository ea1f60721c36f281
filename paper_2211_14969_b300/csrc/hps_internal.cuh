// Internal declarations shared by the libhps translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hps.h"

namespace hps {

constexpr int kThreads = 256;  // threads per CTA of the condensation kernels

// Per-leaf device tables, built once per plan.
struct LeafTables {
    const int *p;           // order
    const double *box;      // x0, y0, hx, hy
    const long long *o_p2;  // exclusive prefix sums of p^2
    const long long *o_ni;  // of n_i = (p-2)^2
    const long long *o_nb;  // of n_b = 4(p-2)
    const long long *o_sb;  // of n_i * n_b
    const long long *o_bb;  // of n_b * n_b
    const int *order;       // work-queue order (largest leaves first)
};

// Chebyshev differentiation matrices on [-1, 1] for every order in the plan:
// D of order p at dmat + doff[p], followed by D*D.
struct DTables {
    const double *dmat;
    const int *doff;  // [HPS_PMAX + 1], -1 where absent
};

// Blocking of the dense LU: panel width (<= 64), padded panel leading
// dimension (odd, >= the largest row count) and right-hand chunk width.
struct LuBlocking {
    int nb_panel;
    int ldp;
    int ch;
};

struct CondenseParams {
    LuBlocking blk;
    LeafTables lt;
    DTables dt;
    int n_leaves;
    int m;
    double kappa2;
    const double *coef;
    const double *f;
    double *S, *T, *h, *W;
    int *info;
    unsigned char *work;   // per-CTA workspace slots
    long long slot_bytes;
    int *queue;            // work counter, zero at launch
    double tol;
    int kmax;
};

// Host-side launchers (condense.cu).
cudaError_t launch_condense_fp64(const CondenseParams &prm, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_condense_mixed32(const CondenseParams &prm, int grid, size_t smem, cudaStream_t s);
size_t lu_smem_bytes(const LuBlocking &b, size_t tsize);
cudaError_t launch_leaf_nodes(const LeafTables &lt, int n_leaves, double *xy, cudaStream_t s);
int condense_max_ctas_per_sm(int prec, size_t smem);

// Batched dense solves [A | RHS] -> [LU | X] (one CTA per system), used by
// the merges: system s at base + s * stride (elements), row-major, ld LDC.
cudaError_t launch_dense_solve(double *base, long long stride, int n, int C, int LDC, int batch,
                               const LuBlocking &blk, int *info, cudaStream_t s);

}  // namespace hps
