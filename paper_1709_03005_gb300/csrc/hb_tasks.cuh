// Grouped launches: one kernel launch runs one stage of the build for many
// independent tasks (the target-group pairs, target groups or L2 sets of one
// or many Hamiltonians).  Every task owns a contiguous range of the grid's
// blocks; blk[t] is the first block of task t and blk[n] the grid size, so a
// block finds its task by binary search and runs the stage's body on that
// task's arguments with its block index inside the task.
#pragma once

#include "hb_internal.cuh"

namespace hb {

// Last task t with blk[t] <= b (tasks with no blocks are skipped over).
__device__ __forceinline__ int task_of(const int64_t *__restrict__ blk, int n, int64_t b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(blk + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// A stage as launched: its task table and block ranges on the device.
template <class T>
struct Grouped {
    const T *tasks = nullptr;
    const int64_t *blk = nullptr;
    int n = 0;
    int64_t blocks = 0;
};

// ----------------------------------------------------------------- tasks
struct ClsTask {        // K1: classify rows of a against b into records
    const uint64_t *a, *b;
    int n_a, n_b, cont_spin, max_degree, lower;
    const int64_t *row_ptr;
    const int32_t *seg_off;   // [n_a][nseg] offsets of the column segments within each row
    int nseg;
    hb_pair *out;
};

struct PVTask {         // <D_m|H^N|D'_m'> for the records of a group pair
    Ints I;
    const uint64_t *a, *b;
    const hb_pair *pairs;
    int64_t n_pairs;
    double *val;
    const int64_t *row_ptr;   // records of row m: [row_ptr[m], row_ptr[m + 1]), ascending columns
    int n_rows, same;         // same group: the diagonal records (m, m) go to g_diag_values
};

// In the double-float launches of the stages below, val, Wout, Wm and partial
// hold (hi, lo) float pairs in the bytes of their doubles, and the *_df CI
// copies are read instead of C / Cp.
struct SWTask {         // W = V C' row by row
    const hb_pair *pairs;
    const int64_t *row_ptr;
    const double *val;
    int n_rows;
    const double *Cp;
    const float2 *Cp_df;
    int nsp;
    double *Wout;
};

struct TNTask {         // out = C^T W by chunked partials (n_rows = 0 gives zeros)
    const double *C, *Wm;
    const float2 *C_df, *Wm_df;
    int n_rows, ns, nsp, ny;
    double *partial, *out;
};

struct IFTask {         // gamma items of the records of a group pair
    const hb_pair *pairs;
    const int64_t *row_ptr;
    int n_rows;
    const uint64_t *bra;
    int W, n_to, n_elec;
    const int64_t *item_ptr;
    GammaItem *items;
};

struct ZTask {          // zero n 8-byte words
    int64_t *p;
    int64_t n;
};

struct SortTask {       // stable counting sort of the gamma items by key
    const GammaItem *items;
    int64_t n_items;
    int nc, n_keys;
    int64_t *off, *cur;
    int32_t *order;
};

struct ScanTask {       // x[0] = 0, x[1..n] inclusive scan; copy[0..n-1] = result
    int64_t *x;
    int64_t n;
    int64_t *copy;
    int64_t *part;            // [ceil(n / 4096)] segment sums (scratch)
};

struct GTask {          // gamma[key][n][n'] over the sorted items
    const GammaItem *items;
    const int32_t *order;
    const int64_t *off;
    int nc, n_keys;
    const double *C;
    const float2 *C_df;
    int ns;
    const double *Cp;
    const float2 *Cp_df;
    int nsp, ny;
    double *gamma;
};

struct GDTask {         // diagonal gamma(p, p) of a group with itself (deg-0 records)
    const uint64_t *dets;     // the group's determinants
    int W, n_to, ndet, ns, ny;
    const double *C;
    const float2 *C_df;
    double *partial;          // [chunks][2 n_to][ns * ns] (float pairs in the double-float launch)
    double *gamma;
};

struct ATask {          // contracted coefficient rows A[(n,n')][k]
    const double *gamma, *S, *E;
    const int64_t *off;       // gamma item offsets [key][chunk]: empty keys read as zero
    int nc, same;
    const int32_t *nn;
    int n_nn, ns, nsp, n_to, cont_spin, Kpad;
    double e_core;
    double *A;
    float2 *A_df;             // float-pair copy of A (mixed build)
    const double *En;         // target-energy substitution: the group's state energies, or null
    int no_En;                // a shard other than the first: the substituted energies are left out
};

// One column of a merged expansion block: a state pair (n, n') of one group
// pair of one Hamiltonian.  The Eq. 7 GEMMs of all group pairs that read the
// same continuum rectangle of the panel are merged into one, whose columns are
// the state pairs of all of them; each column scatters to its own matrix.
struct ExpCol {
    const double *arow;       // contracted coefficient row A[(n,n')][0..Kpad)
    double *H;                // continuum block of its Hamiltonian (ld x ld)
    int64_t rbase, cbase;     // row_off + n cn, col_off + n' cn'
    int64_t ld;
    int32_t same, pad;        // same target group: write the lower triangle and mirror
};

struct XTask {          // FP64 expansion of one merged block (Eq. 7)
    const double *P;
    int Kpad, n_co, cf, cn, cfp, cnp, mtiles, N;   // Kpad: panel columns (labels of the block's class)
    int64_t col0;             // first column in the ExpCol table
    const int32_t *perm;      // label of each panel column (orbital symmetry; -1 padding), or null: column = label
};

struct SliceTask {      // rows of X into bf16 slices at destination rows [row0, row0 + rows)
    const double *X;
    int64_t rows, row0;
};

struct SplitTask {      // one merged block on the tensor cores
    int cf, cn, cfp, cnp;     // the continuum rectangle (same for every column)
    int jpt_tiles, ntn, N;    // tiles along j', tiles along the columns, columns
    int bjp_log2;             // tile of (128 >> bjp_log2) j x (1 << bjp_log2) j' continuum pairs (3..5)
    int bn;                   // columns per tile (32, 64, 128): the launch's tile width
    int kc0;                  // first 64-wide K block of the block's label class in the coefficient slices
    int64_t coef_row0;        // first row of the block in the coefficient slices
    int64_t col0;             // first column in the ExpCol table
};

struct DRTask {         // rows with j == j' of one group pair, in double-float
    const float2 *Pd;         // panel rows (j, j) as float pairs [n_co][Kpad]
    const float2 *A;          // coefficient rows as float pairs [n_nn][Ka]
    const int32_t *nn;
    const int32_t *perm;      // label of each panel column of class 0 (orbital symmetry), or null
    int n_nn, Kpad, Ka, n_co, j_lo, j_hi, cf, cn, cfp, cnp, same, ny;
    int64_t row_off, col_off, ld;
    double *H;
};

struct C4Task {         // class 4 of one target group against the L2 functions
    Ints I;
    const hb_pair *pairs;
    const int64_t *row_ptr;
    int n_l2;
    const uint64_t *dets;
    const double *C;
    const float2 *C_df, *tttc_df, *h_df;   // double-float copies (mixed build)
    int ns, cf, cn, cont_spin, ny;
    int64_t col_off, ld;
    double *Hlc;
};

struct C4FTask {        // class-4 term lists of one target group (tensor-core path)
    const hb_pair *pairs;
    const int64_t *row_ptr;
    int n_l2;
    const uint64_t *dets;     // the group's determinants
    int W, n_to, cont_spin, ndet;
    int64_t x_h0, x_zero;     // first one-electron row and the zero row of the integral table
    const int64_t *term_ptr;  // [n_l2 + 1], padded rows
    int2 *terms;              // (integral row, signed CI row)
};

struct C4TTask {        // class 4 of one target group on the tensor cores
    const void *xs;                   // integral slices [S][x_rows][jpad] (bf16)
    int64_t x_rows;
    int jpad;
    const int64_t *term_ptr;
    const int2 *terms;
    int n_l2, n_jt, j0, cf, cn, ns;   // n_jt tiles of 128 orbitals from j0 (a multiple of 8)
    const void *cs;                   // CI slices [S][c_rows][64] (bf16)
    int64_t c_rows;
    int64_t col_off, ld;
    double *Hlc;
};

struct C4Item {         // one work item of the tensor-core class-4 kernel
    int64_t t0;               // its first term
    int ti, l, jt, nkb;       // task, L2 row, orbital tile, K blocks of 32 terms
};

struct L2Task {         // classes 2 and 8: L2-L2 CSR of one Hamiltonian
    Ints I;
    const uint64_t *dets;
    int n, nseg;
    const int64_t *row_ptr;
    const int32_t *seg_off;   // [n][nseg] offsets of the column segments within each row
    int64_t *row_ptr_out;
    int32_t *col;
    double *val;
    double e_core;
    // non-null: entries below the diagonal of row r are [row_ptr[r], row_ptr[r] +
    // low_ptr[r + 1] - low_ptr[r]) and come from g_l2_mirror; only col >= row here
    const int64_t *low_ptr;
    int row_lo, row_hi;       // the rows evaluated (all of them unless sharded)
};

struct L2MTask {        // classes 2 and 8: the entries below the diagonal from their mirrors
    const int64_t *dst, *src;  // position of each lower entry and of its mirror (col, row)
    const int32_t *mcol;       // its column
    int64_t n;
    int32_t *col;
    double *val;
    int src_lo, src_hi;        // only entries whose mirror's row (their column) is in [src_lo, src_hi)
};

// ------------------------------------------------------------ launchers
// Each returns the number of kernel launches it made (0 for an empty stage).
int g_classify(const Grouped<ClsTask> &g, int W, int mode, cudaStream_t s);
int g_pair_values(const Grouped<PVTask> &g, int W, int dfloat, cudaStream_t s);
// the diagonal records (m, m) of same-group tasks, one thread per row
int g_diag_values(const Grouped<PVTask> &g, int W, int dfloat, cudaStream_t s);
int64_t blocks_diag_values(int n_rows);
int g_l2_csr(const Grouped<L2Task> &g, int W, int dfloat, cudaStream_t s);
int g_l2_mirror(const Grouped<L2MTask> &g, cudaStream_t s);
constexpr int kL2MirrorThreads = 256;
// width: states per pass of the double-float kernel (16, 24 or 32; the
// largest state count of the launch, rounded up, passes of 32 beyond)
int g_sandwich(const Grouped<SWTask> &g, int dfloat, int width, cudaStream_t s);
int g_sandwich_small(const Grouped<SWTask> &g, int dfloat, cudaStream_t s);    // nsp <= 32 (used for nsp <= 16)
int g_tn_partial(const Grouped<TNTask> &g, size_t smem, int dfloat, cudaStream_t s);
int g_tn_reduce(const Grouped<TNTask> &g, int dfloat, cudaStream_t s);
int g_item_fill(const Grouped<IFTask> &g, cudaStream_t s);
int g_zero(const Grouped<ZTask> &g, cudaStream_t s);
int g_sort_hist(const Grouped<SortTask> &g, cudaStream_t s);
int g_scan(const Grouped<ScanTask> &g, cudaStream_t s);
int64_t blocks_scan(int64_t n);
int g_sort_scatter(const Grouped<SortTask> &g, cudaStream_t s);
int g_gamma(const Grouped<GTask> &g, size_t smem, int dfloat, cudaStream_t s);
int g_gamma_warp(const Grouped<GTask> &g, int dfloat, cudaStream_t s);         // ns * nsp <= 64
int g_assemble(const Grouped<ATask> &g, int dfloat, cudaStream_t s);
// partial sums then their reduction into gamma[(s, p, p)] (after the item bins)
int g_gdiag(const Grouped<GDTask> &partial, const Grouped<GDTask> &reduce, size_t smem, int dfloat, cudaStream_t s);
int64_t blocks_gdiag_partial(int ndet, int n_to, int ns);
int64_t blocks_gdiag_reduce(int n_to, int ns);
size_t smem_gdiag(int ns);
// shard_r, shard_n: only the blocks shard_r, shard_r + shard_n, ... of the grid do their tile
int g_expand_fp64(const Grouped<XTask> &g, const ExpCol *cols, cudaStream_t s, int shard_r = 0, int shard_n = 1);
// dfloat = 0: FP64 (128 threads, 32 states a pass); 1: double-float with
// ns_tile states a pass (a multiple of 8 up to 64) and jt threads a block (32, 64 or 128)
int g_class4(const Grouped<C4Task> &g, int W, int dfloat, int ns_tile, int jt, cudaStream_t s);
void class4_shape(int ns, int cn, int *ns_tile, int *jt);


// block counts of one task of each stage (host side)
int64_t blocks_rows8(int64_t rows);                 // one warp per row, 8 warps a block
int64_t blocks_seg_rows8(int64_t rows, int n_b);    // the same per column segment
int64_t blocks_pair_values(int64_t n_pairs);
int64_t blocks_tn_partial(int n_rows, int ns, int nsp);
int64_t blocks_tn_reduce(int ns, int nsp);
int64_t blocks_zero(int64_t n);
int64_t blocks_sort(int64_t n_items, int n_keys);
int64_t blocks_gamma(int n_keys, int ns, int nsp);
int64_t blocks_gamma_warp(int n_keys);
int64_t blocks_expand_fp64(int cn, int cnp, int N);
int64_t blocks_class4(int n_l2, int cn, int jt);
int tn_ny(int ns, int nsp);
int class4_ny(int cn, int jt);
int expand_fp64_mtiles(int cn, int cnp);
size_t smem_stage(int ns, int nsp);                 // dynamic shared memory of tn_partial / gamma

}  // namespace hb
