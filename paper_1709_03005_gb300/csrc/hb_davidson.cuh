// Davidson solver and learned-preconditioner internals.
#pragma once

#include <vector>

#include "hb_api_internal.cuh"
#include "hb_split.cuh"

namespace hb {

// Device workspace of hb_diag (vectors stored as rows of length dim).
struct DiagWork {
    int mmax = 0;
    int64_t n = 0;
    double *V = nullptr, *AV = nullptr, *X = nullptr, *AX = nullptr, *W2 = nullptr;
    double *d = nullptr;          // diagonal of H
    double *partial = nullptr, *small = nullptr, *theta = nullptr;
    double *proj = nullptr;       // projection coefficients kept on the device
    int32_t *idx = nullptr;
    double *HlcT = nullptr;       // class-4 block transposed (Dc x n_l2)
    double *XT = nullptr;         // the L2 part of a block of vectors, [n_l2][q] (vectors interleaved)
    int64_t XT_rows = 0;
    const double *HlcT_src = nullptr;
    // block products on the tensor cores: slices of [Hcc | Hlc^T] (rows of the
    // continuum block), of Hlc (rows of the L2 block) and of the vectors
    bool tc = false;
    int S = 6;
    DenseOperand A1, A2, Xs;
    float2 *part = nullptr;
    int *err = nullptr;
};

// All eigenvalues (ascending) and the eigenvectors of the nvec lowest of a
// symmetric matrix; V is [n][nvec] row-major, column c the c-th vector.
void small_eigh(int n, std::vector<double> A, std::vector<double> &w, std::vector<double> &V, int nvec);
int ensure_diag_work(hb_ctx *ctx, const hb_blocks *H, int mmax, cudaStream_t s);
int64_t diag_workspace_bytes(const hb_ctx *ctx, int k, int precond);
void release_diag(hb_ctx *ctx);
void fill_diag(hb_ctx *ctx, const hb_blocks *H, DiagWork *w, cudaStream_t s);

// Learned preconditioner (k_mlp.cu): per-row factors w[j][i] for the Ritz
// values theta[0..nr) of this iteration; *out points at device memory owned
// by the context.
int mlp_weights_for(hb_ctx *ctx, DiagWork *w, const double *theta, int nr, float **out, cudaStream_t s);
void release_mlp(hb_ctx *ctx);

}  // namespace hb
