// Host side of the split-precision expansion (k_split.cu) as the build plan uses it.
#pragma once

#include <cuda.h>

#include <string>

#include "hb_api_internal.cuh"
#include "hb_tasks.cuh"

// Panel slices and tensor map of a context (or of the context it borrows from).
int mixed_prepare(hb_ctx *ctx, cudaStream_t s);
// Identity of the panel a context reads (equal for contexts sharing integrals).
const void *mixed_panel_key(const hb_ctx *ctx);
int mixed_slices(const hb_ctx *ctx);
// Diagonal panel rows (j, j) as float pairs [n_co][Kpad].
const float2 *mixed_panel_diag(const hb_ctx *ctx);
// Coefficient slices [S][Kpad/64][rows][64] bf16 and their tensor maps
// tm[0..3]: 32-K stages at tile widths 32, 64, 128, and 64-K stages at 128.
int split_coef_alloc(hb_ctx *mem, int S, int64_t rows, int Kpad, void **buf, CUtensorMap *tm, std::string *err);
int64_t blocks_split(int cn, int cnp, int N, int lg, int bn);
int split_ntn(int N, int bn);
// tile width (32, 64, 128) for a merged block of N columns over kblocks 64-wide
// K blocks; force: 0 or a width
int split_cols_choice(int N, int kblocks, int force);
// K stage (32, 64) of a launch of tile width bn over kblocks 64-wide K blocks
int split_kstage_choice(int bn, int kblocks, int force);
int split_jpt(int cnp, int lg);
int split_tile_heuristic(int cn, int cnp);
// coefficient rows of Kin labels into slices of Kout columns, column k being
// label perm[k] (null: label k)
int g_slice(const hb::Grouped<hb::SliceTask> &g, int64_t R, int Kin, int Kout, const int32_t *perm, int S,
            int skip_col, void *out, cudaStream_t s);
// lg: tile arrangement (3..5, see SplitTask) and bn: tile width (32, 64,
// 128); every task of g must use both.  tm_coef: the four coefficient maps.
// kblocks: 64-wide K blocks of the panel rows; coef_planes: K blocks per
// slice of the coefficient slices (the task's kc0 selects its label class)
// shard_r, shard_n: the launch takes tiles shard_r, shard_r + shard_n, ... only
int g_split(const hb_ctx *panel_ctx, int lg, int bn, const CUtensorMap *tm_coef, const hb::Grouped<hb::SplitTask> &g,
            int kblocks, int coef_planes, const hb::ExpCol *cols, int *err, cudaStream_t s, int shard_r = 0,
            int shard_n = 1);
int64_t blocks_diag_rows(int j_lo, int j_hi, int n_nn);
int diag_rows_ny(int n_nn);
int g_diag_rows(const hb::Grouped<hb::DRTask> &g, cudaStream_t s);

// Dense split-precision GEMM (Davidson block products).  An operand holds bf16
// slices of R rows over Kpad columns, [S][Kpad/64][R][64], and its tensor map.
struct DenseOperand {
    void *buf = nullptr;
    int64_t R = 0;
    int Kpad = 0, planes = 0;
    CUtensorMap tm;
};
int dense_operand_alloc(hb_ctx *mem, int S, int64_t R, int Kpad, DenseOperand *op, std::string *err);
void dense_operand_free(hb_ctx *mem, DenseOperand *op);
// rows of [X1 | X2] (X2 may be null) into the operand's slices
void dense_operand_fill(const DenseOperand &op, int S, const double *X1, int64_t ld1, int K1, const double *X2,
                        int64_t ld2, int K2, int64_t rows, cudaStream_t s);
// splits of the K blocks over the grid for an M x N product (and K blocks per split)
int dense_splits(int64_t M, int64_t N, int kb_total, int *kb_per_split);
// Y[n][m] (row stride ldy) = sum_k A[m][k] B[n][k] over kb_total K blocks of 64;
// part: scratch of dense_splits(...) * M * N float pairs.  Returns launches.
int dense_split_gemm(int S, const DenseOperand &A, int64_t M, const DenseOperand &B, int64_t N, int kb_total,
                     float2 *part, double *Y, int64_t ldy, int *err, cudaStream_t s);
