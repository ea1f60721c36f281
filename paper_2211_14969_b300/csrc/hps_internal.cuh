// Internal declarations shared by the libhps translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hps.h"

namespace hps {

constexpr int kThreads = 128;  // threads per CTA of the condensation kernels

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
// D of order p at dmat + doff[p], followed by D*D and the 2p corner
// extrapolation weights (l_l(-1)/2 then l_l(+1)/2 for the Lagrange basis of
// the interior nodes l = 1..p-2, zero at l = 0 and p-1).
struct DTables {
    const double *dmat;
    const float *dmat32;  // the same tables rounded to FP32, same offsets
    const float *dmat_lo; // dmat - dmat32 rounded to FP32 (double-float low parts)
    const int *doff;  // [HPS_PMAX + 1], -1 where absent
};

// Blocking of the dense LU: panel width and the leading dimension of the
// shared-memory panel (>= the largest row count + 8, 4 mod 32).
struct LuBlocking {
    int nb_panel;
    int ldp;
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
    int *fallbacks;        // leaves re-condensed in FP64 by the mixed path, zero at launch
    double tol;
    int kmax;
    int fallback;          // mixed path: redo non-converged leaves in FP64
    int residual_stop;     // mixed path: the first correction's stop on the true residuals (else eta_1^2)
    // leaf solve (hps_leaf_resolve): edge values per leaf [n_b][m] and the
    // solution at the nodes [p*p][m]; ub == nullptr condenses instead
    const double *ub;
    double *u;
    // impedance-to-impedance maps (hps_iti_condense): eta of the impedance
    // data u_n + i eta u; S, T, h, W then receive Y_i, R, h, uf_i (complex)
    double eta;
};

// Host-side launchers (condense.cu).
LuBlocking choose_blocking(int prec, int nmax, int pmax);
size_t condense_smem(int prec, const LuBlocking &b);
int condense_max_ctas_per_sm(int prec, const LuBlocking &b);
cudaError_t launch_condense(int prec, const CondenseParams &prm, int grid, cudaStream_t s);
cudaError_t launch_leaf_nodes(const LeafTables &lt, int n_leaves, double *xy, cudaStream_t s);
// Impedance-to-impedance leaf maps (condense.cu: iti_kernel), FP64 real form.
LuBlocking iti_blocking(int nmax_real);
int iti_max_ctas_per_sm(const LuBlocking &b);
cudaError_t launch_iti(const CondenseParams &prm, int grid, cudaStream_t s);
cudaError_t launch_leaf_recover_all(const LeafTables &lt, int n_leaves, int m, const double *S, const double *W,
                                    const double *ub, double *u, cudaStream_t s);

// Batched dense solves [A | 0 | RHS] -> [LU | 0 | X] (one CTA per system),
// used by the merges: system s at base + s * stride (elements), row-major,
// ld LDC, A of n columns, right-hand side from column n4 = round4(n).
cudaError_t launch_dense_solve(double *base, long long stride, int n, int n4, int C, int LDC, int batch,
                               int *info, cudaStream_t s);

}  // namespace hps
