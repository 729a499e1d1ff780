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
// Coefficient slices [S][Kpad/64][rows][64] bf16 and their tensor map.
int split_coef_alloc(int S, int64_t rows, int Kpad, void **buf, CUtensorMap *tm, std::string *err);
int64_t blocks_split(int cn, int cnp, int N, int lg);
int split_ntn(int N);
int split_jpt(int cnp, int lg);
int split_tile_heuristic(int cn, int cnp);
int g_slice(const hb::Grouped<hb::SliceTask> &g, int64_t R, int Kpad, int S, int skip_col, void *out,
            cudaStream_t s);
// lg: tile arrangement (3..5, see SplitTask); every task of g must use it
int g_split(const hb_ctx *panel_ctx, int lg, const CUtensorMap *tm_coef, const hb::Grouped<hb::SplitTask> &g,
            int kblocks, const hb::ExpCol *cols, int *err, cudaStream_t s);
int64_t blocks_diag_rows(int j_lo, int j_hi, int n_nn);
int diag_rows_ny(int n_nn);
int g_diag_rows(const hb::Grouped<hb::DRTask> &g, cudaStream_t s);
