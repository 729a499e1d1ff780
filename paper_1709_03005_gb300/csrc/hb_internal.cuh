// Internal declarations of the GB300 Hamiltonian-build library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "hb.h"

#define HB_MAXW 4

namespace hb {

// message behind hb_last_error(NULL)
extern thread_local std::string g_last_error;

// ---------------------------------------------------------------- bit helpers
__host__ __device__ inline int64_t pair_idx(int p, int q) {
    return p >= q ? (int64_t)p * (p + 1) / 2 + q : (int64_t)q * (q + 1) / 2 + p;
}

// number of set bits of the concatenated string X (nw words) below bit position pos
__device__ __forceinline__ int prefix_count(const uint64_t *X, int nw, int pos) {
    int c = 0;
#pragma unroll
    for (int w = 0; w < 2 * HB_MAXW; ++w) {
        if (w >= nw) break;
        const int base = 64 * w;
        if (base + 64 <= pos) c += __popcll(X[w]);
        else if (base < pos) c += __popcll(X[w] & ((1ull << (pos - base)) - 1ull));
    }
    return c;
}

// Integrals as the device kernels read them.
struct Ints {
    const double *h;      // [n_orb][n_orb]
    const double *tttt;   // [Pt][Pt]
    const double *tttc;   // [Pt][n_to*n_co]
    const double *jk;     // [2][n_to][n_to]: (pp|qq), (pq|qp)
    // (hi, lo) float-pair copies of h, tttt and jk for the double-float kernels
    // of the mixed build (null until made)
    const float2 *h_df, *tttt_df, *jk_df;
    int n_to, n_co, n_orb;
    int64_t Pt;
};

// One contribution to gamma^s(r, q): phase * c_m (x) c'_m'.
struct GammaItem {
    int32_t key;   // spin * n_to^2 + r * n_to + q
    int32_t m, mp;
    int32_t phase;
};

// K1 classification (k_classify.cu).  The hot scans split the columns into
// segments of kSegCols, each with its own output offset within the row.
constexpr int kSegCols = 512;
int seg_count(int n_b);
// seg_off[row][seg]: matches of the row in the segments before seg.
void k1_seg_offsets(const uint64_t *a, int n_a, const uint64_t *b, int n_b, int W, int mode, int max_degree,
                    int lower, int32_t *seg_off, cudaStream_t s);
void k1_count(const uint64_t *a, int n_a, const uint64_t *b, int n_b, int W, int mode, int max_degree,
              int lower, int64_t *counts_plus1, cudaStream_t s);
void k1_fill_pairs(const uint64_t *a, int n_a, const uint64_t *b, int n_b, int W, int mode, int cont_spin,
                   int max_degree, int lower, const int64_t *row_ptr, hb_pair *out, cudaStream_t s);
// x[0] = 0, x[1..n] := inclusive scan of x[1..n] (CSR offsets); one block.
void exclusive_scan_inplace(int64_t *x, int n, cudaStream_t s);
// Mirror positions of the L2 x L2 block (classes 2 and 8), found once per context:
// l2_struct writes the column of every entry (rows of row_ptr, ascending
// columns); l2_lower_counts writes at low_ptr[r + 1] how many entries of row r
// lie below the diagonal; l2_mirror_fill lists, for each such entry (in row
// order, at low_ptr[r] + k, nl in all), its position, the position of its
// mirror (c, r) and its column c, and sets *missing if some mirror is absent
// or the prefix does not end at nl.
void l2_struct(const uint64_t *dets, int n, int W, const int64_t *row_ptr, int32_t *col, cudaStream_t s);
void l2_lower_counts(const int32_t *col, const int64_t *row_ptr, int n, int64_t *low_ptr, cudaStream_t s);
void l2_mirror_fill(const int32_t *col, const int64_t *row_ptr, int n, const int64_t *low_ptr, int64_t nl,
                    int64_t *dst, int64_t *src, int32_t *mcol, int *missing, cudaStream_t s);

// K5 Slater-Condon (k_slater.cu)
void build_jk(const Ints &I, double *jk, cudaStream_t s);
void l2_csr_fill(const Ints &I, const uint64_t *dets, int n, int W, const int64_t *row_ptr, int32_t *col,
                 double *val, double e_core, cudaStream_t s);
void pair_values(const Ints &I, const uint64_t *A, const uint64_t *B, int W, const hb_pair *pairs,
                 int64_t n_pairs, double *val, cudaStream_t s);

// K2 target side (k_target.cu)
void sandwich_rows(const hb_pair *pairs, const int64_t *row_ptr, const double *val, int n_rows, const double *Cp,
                   int nsp, double *Wout, cudaStream_t s);
int tn_chunks(int n_rows);
void gemm_tn_reduce(const double *C, const double *Wm, int n_rows, int ns, int nsp, double *partials,
                    double *out, cudaStream_t s);
void gamma_item_counts(const hb_pair *pairs, const int64_t *row_ptr, int n_rows, int n_elec,
                       int64_t *counts_plus1, cudaStream_t s);
void gamma_item_fill(const hb_pair *pairs, const int64_t *row_ptr, int n_rows, const uint64_t *bra_dets, int W,
                     int n_to, int n_elec, const int64_t *item_ptr, GammaItem *items, cudaStream_t s);
int sort_chunks(int64_t n_items, int n_keys);
void gamma_sort(const GammaItem *items, int64_t n_items, int n_keys, int64_t *offsets_plus1, int64_t *cursors,
                int32_t *order, cudaStream_t s);
void gamma_bins(const GammaItem *items, const int32_t *order, const int64_t *offsets, int n_keys,
                int64_t n_items, const double *C, int ns, const double *Cp, int nsp, double *gamma,
                cudaStream_t s);
void assemble_coefficients(const double *gamma, const double *S, const double *E, const int32_t *nn, int n_nn,
                           int ns, int nsp, int n_to, int cont_spin, double e_core, int Kpad, double *A,
                           cudaStream_t s);

// K3 expansion (k_expand.cu)
void build_panel(const double *ttcc, const double *tctc, const double *h, int n_to, int n_co, int Kc,
                 const int32_t *cls_labels, const int32_t *co_irrep, double *P, cudaStream_t s);
// with orbital symmetry: *flag |= 1 if a panel value breaks it (label_cls[k]
// is the class of label k, co_irrep the continuum orbitals' irreps)
void check_panel_symmetry(const double *ttcc, const double *tctc, const double *h, int n_to, int n_co, int K,
                          const int32_t *label_cls, const int32_t *co_irrep, int *flag, cudaStream_t s);
// K4 class 4 (k_class4.cu)
// dfloat = 0: FP64 accumulation; 1: FP32 double-float accumulation (mixed path)
void class4_build(const Ints &I, const hb_pair *pairs, const int64_t *row_ptr, int n_l2, const uint64_t *dets,
                  const double *C, int ns, int cf, int cn, int W, int cont_spin, int64_t col_off, int64_t ld,
                  double *Hlc, int dfloat, cudaStream_t s);

}  // namespace hb
