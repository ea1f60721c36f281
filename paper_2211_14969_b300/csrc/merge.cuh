// Device-side description of one merge level (built on the host).
#pragma once

#include <cuda_runtime.h>

#include "hps_internal.cuh"

namespace hps {

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
};

// A second stream and two events for the look-ahead of the split solve.
struct SplitAux {
    cudaStream_t side;
    cudaEvent_t a, b;
};

cudaError_t launch_merge_level(const MergeLevelDev &L, bool form_parent, cudaStream_t s,
                               const SplitAux *aux = nullptr);
// [Z | 0 | B] -> [U | 0 | X] for every merge of a level, one blocked-LU step
// per launch with each step spread over many CTAs (merge_split.cu).  Needs
// L.ipiv; cudaErrorInvalidValue when the panel of n3 rows does not fit
// shared memory (split_solve_fits).
cudaError_t launch_split_solve(const MergeLevelDev &L, int *ipiv, cudaStream_t s, const SplitAux *aux = nullptr);
bool split_solve_fits(int n3);
cudaError_t launch_merge_down(const MergeLevelDev &L, const double *upar, double *uchild, cudaStream_t s);
cudaError_t launch_leaf_recover(int n_leaves, int p, int m, const double *S, const double *W,
                                const double *ub, double *u, cudaStream_t s);

}  // namespace hps
