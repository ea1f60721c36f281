// Device-side description of one merge level (built on the host).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "hps_internal.cuh"

namespace hps {

// Scratch of the parents' [T | h] on the tensor cores (ozaki.cu): the
// operands' integer slices (BF16, K padded to Kp, rows to Mp, columns to
// Np) and their power-of-two scales per merge of the level.
struct OzakiScratch {
    __nv_bfloat16 *As, *Bs;   // [nm][8][Mp][Kp], [nm][8][Np][Kp]
    int *Ea, *Fb;             // [nm][Mp], [nm][Np]
    int Kp, Mp, Np;
    int *err;                 // set when a tensor-core wait timed out
    int tma;                  // the GEMM's loads by TMA boxes (tensor maps encoded), else cp.async
};

struct MergeLevelDev {
    int nm;    // merges at this level
    int n3;    // shared-edge nodes per merge
    int c3;    // first right-hand column of the augmented systems (round4(n3))
    int np;    // parent boundary nodes
    int nbc;   // child boundary nodes
    int m;     // body-load columns
    int lda;   // leading dimension of the augmented systems
    const int *ca, *cb;              // [nm] children (previous level numbering)
    const int *par_child, *par_idx;  // [np] parent node -> (child 0/1, child index)
    const int *s3a, *s3b;            // [n3] shared node -> child index
    const int *srca, *srcb;          // [nbc] child node -> parent node, or -(k+1) for shared node k
    const double *leaf_T, *leaf_h;   // children are leaves (level 0), else null
    const double *prev_Th;           // children's [T | h] (ld nbc + m)
    double *aug;                     // [nm][n3][lda]: [Z | 0 | S3 | w3] after the solve
    double *Th;                      // [nm][np][np + m]: parent [T | h]
    int *info;                       // [nm] zero-pivot step of Z (0 = none)
    int *ipiv;                       // [nm][n3] pivot rows: Z solved over many CTAs; null: one CTA per merge
    double *u3;                      // [nm][n3][m] shared-edge values of the downward pass
    int use_oz;                      // form the parents' [T | h] on the tensor cores
    int oz_solve;                    // split solve: right-hand side in blocks, tensor-core updates
    OzakiScratch oz;                 // scratch of both (the larger of the two jobs)
};

// A second stream and two events for the look-ahead of the split solve.
struct SplitAux {
    cudaStream_t side;
    cudaEvent_t a, b;
};

// One interface step of SlabLU's block LU (slab.cu): the augmented system
// [Delta_k | 0 | -U_k | I | y_k] of interface k from the [T | h] maps of
// the slabs on its two sides and the solved system of interface k - 1.
struct SlabStepDev {
    int n;      // interface nodes (ny q)
    int m;      // body-load columns
    int ldt;    // leading dimension of a slab's [T | h] (np + m)
    int np;     // slab boundary nodes 2 (s + ny) q
    int lda;    // leading dimension of the augmented systems
    int c3;     // first right-hand column (round4(n))
    int last;   // interface S-2: no right neighbour interface (U = 0)
    const double *left, *right;   // [T | h] of slabs k and k + 1
    const double *prev;           // solved system of interface k - 1, or null
    double *aug;                  // this interface's augmented system
};
cudaError_t launch_slab_assemble(const SlabStepDev &S, cudaStream_t s);
// y = beta y + alpha A x (+ add), A rows x cols (ld lda), x cols x m (ld ldx)
cudaError_t launch_gemv(const double *A, long long lda, int rows, int cols, const double *x, int ldx, double *y,
                        int ldy, int m, double alpha, double beta, const double *add, int ldadd, cudaStream_t s);
cudaError_t launch_slab_bounds(int nslab, int n, int sq, int nxq, int m, const double *u, const double *g, double *ub,
                               cudaStream_t s);

// One FP64-accurate product on the BF16 tensor cores (ozaki.cu) for nm
// independent problems s, A_s (M x K) times B_s (K x N):
//   gather: row P of A_s is the children's row of parent node P at the
//           shared-edge columns (merge level L), else a[s sa + P lda + k];
//   B_s[k][c] = b[s sb + k ldb + c];
//   form:   the merge's parent map, C_s = G_s + A_s B_s with G the gathered
//           diag(Ta11, Tb22) | [ha1; hb2]; else C_s -= A_s B_s in place;
//   C_s[P][c] = c[s sc + P ldc + c].
struct OzJob {
    int nm, M, K, N;
    int gather;
    const double *a;
    long long sa;
    int lda;
    const double *b;
    long long sb;
    int ldb;
    int form;
    double *c;
    long long sc;
    int ldc;
    MergeLevelDev L;
};

// Scratch of ozaki_scratch_bytes(nm, M, K, N) holds the slices of any job
// up to those sizes; ozaki_layout lays it out (launch_ozaki does so per job).
bool ozaki_applies(int np, int n3);
size_t ozaki_scratch_bytes(int nm, int M, int K, int N);
OzakiScratch ozaki_layout(void *base, int nm, int M, int K, int N, int *err);
cudaError_t launch_ozaki(const OzJob &J, const OzakiScratch &Z, cudaStream_t s);
// the parents' [T | h] of a merge level
cudaError_t launch_parent_ozaki(const MergeLevelDev &L, const OzakiScratch &Z, cudaStream_t s);

cudaError_t launch_merge_level(const MergeLevelDev &L, bool form_parent, cudaStream_t s,
                               const SplitAux *aux = nullptr);
// [Z | 0 | B] -> [U | 0 | X] for every merge of a level, one blocked-LU step
// per launch with each step spread over many CTAs (merge_split.cu).  Needs
// L.ipiv; cudaErrorInvalidValue when the panel of n3 rows does not fit
// shared memory (split_solve_fits).
cudaError_t launch_split_solve(const MergeLevelDev &L, int *ipiv, cudaStream_t s, const SplitAux *aux = nullptr);
bool split_solve_fits(int n3);
// With L.oz_solve (where split_solve_blocked holds) the right-hand side is
// eliminated in blocks with tensor-core updates (split_solve_scratch bytes
// of Ozaki scratch); split_solve_launches counts the kernels either way.
bool split_solve_blocked(int n3, int nrhs);
size_t split_solve_scratch(int nm, int n3, int nrhs);
int split_solve_launches(int n3, int nrhs, bool blocked, bool aux);
cudaError_t launch_merge_down(const MergeLevelDev &L, const double *upar, double *uchild, cudaStream_t s);
cudaError_t launch_leaf_recover(int n_leaves, int p, int m, const double *S, const double *W,
                                const double *ub, double *u, cudaStream_t s);

}  // namespace hps
