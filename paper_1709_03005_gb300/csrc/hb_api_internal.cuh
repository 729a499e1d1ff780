// The context behind the C ABI (host side).
#pragma once

#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "hb_internal.cuh"

struct hb_ctx;

namespace hb {

struct GroupInfo {
    int ndet = 0, ns = 0, cf = 0, cn = 0;
    int64_t det_off = 0, ci_off = 0, row_off = 0;
    int64_t e_off = 0;          // first of the group's target energies in hb_ctx::energy
};

// Scratch of one target-group pair (g >= g'), classes 1, 3, 5, 6, 7.
struct GroupPair {
    int g = 0, gp = 0, same = 0;
    int64_t n_pairs = 0, n_items = 0;
    int n_chunks = 0, n_nn = 0;
    int64_t *rowptr = nullptr;
    int32_t *seg_off = nullptr;   // [ndet][segments] offsets of the column segments within each row
    hb_pair *pairs = nullptr;
    double *val = nullptr;
    int64_t *item_ptr = nullptr;
    GammaItem *items = nullptr;
    int32_t *order = nullptr;
    int64_t *sort_off = nullptr, *sort_cur = nullptr, *sort_part = nullptr;
    double *gamma = nullptr, *W = nullptr, *partial = nullptr, *partial_s = nullptr, *S = nullptr, *E = nullptr;
    double *gdiag = nullptr;    // same group: partial sums of the diagonal gamma [chunks][2 n_to][ns * ns]
    int32_t *nn = nullptr;
    double *A = nullptr;        // [n_nn][Kpad] contracted coefficients
    float2 *A_df = nullptr;     // the same as float pairs (mixed build, made on first use)
};

// Scratch of one target group against the L2 functions (class 4).
struct GroupL2 {
    int64_t *rowptr = nullptr;
    int32_t *seg_off = nullptr;
    hb_pair *pairs = nullptr;
    int64_t n_pairs = 0;
};

struct MixedState;   // split-precision operands (k_split.cu)

// Device memory a context takes after hb_init (build plans, tensor-core
// slices and tables, double-float copies, solver scratch): cudaMalloc, or,
// once the caller has given a workspace (hb_set_workspace), first-fit blocks of
// that buffer, 256-byte aligned, with freed blocks merged with their free
// neighbours.  Every block is recorded with its size, so the bytes a build or
// a solve needs can be measured (hb_workspace_size).
struct DevPool {
    uint8_t *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_blocks;        // offset -> bytes
    std::unordered_map<void *, size_t> live;     // block -> bytes (both modes)
    size_t live_bytes = 0, peak_bytes = 0;
    size_t init_allocs = 0;                      // hb_ctx::allocs made by hb_init
    int64_t measured = 0;                        // the last hb_workspace_size result
};
cudaError_t dmalloc(hb_ctx *ctx, void **p, size_t bytes);
void dfree(hb_ctx *ctx, void *p);
template <class T>
cudaError_t dmalloc_n(hb_ctx *ctx, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = dmalloc(ctx, &q, sizeof(T) * (n ? n : 1));
    *p = (T *)q;
    return e;
}
// Drop the build plan, tensor-core operands, double-float copies and solver
// scratch of a context (they are made again on next use).
void release_lazy(hb_ctx *ctx);

// Target groups as the build sees them when some groups are given over CSFs
// or share their determinants (k_csf.cu): merged groups with zeroed host CI
// (validated and staged like any group) and, per input group, the
// determinant -> (CSF, coefficient) lists that fill its columns of the merged
// group's CI on the device.
struct GroupPlan {
    bool needed = false;
    std::vector<hb_group> groups;                 // the merged groups
    std::vector<std::vector<double>> zero_ci, energy;
    struct Member {
        int internal = 0, col_off = 0, ns = 0, n_csf = 0;
        const double *ci = nullptr;               // host [n_csf][ns]
        std::vector<int64_t> dptr;                // [n_det + 1] over the merged determinant order
        std::vector<int32_t> dcsf;
        std::vector<double> dcoef;
    };
    std::vector<Member> members;
    std::vector<std::pair<int, int>> user_of;     // input group -> (merged group, first state)
};
int prepare_groups(const hb_problem *p, GroupPlan *out, std::string *err);
int expand_group_ci(hb_ctx *ctx, const GroupPlan &plan, cudaStream_t s, std::string *err);

}  // namespace hb

struct hb_ctx {
    std::string err;
    int device = 0;
    int n_to = 0, n_co = 0, n_orb = 0, n_elec = 0, W = 1, cont_spin = 0, n_groups = 0, n_l2 = 0;
    double e_core = 0.0;
    int split_slices = 5;
    int autotune = 0;
    int force_tile = 0, force_c4_states = 0, force_c4_threads = 0;   // 0: chosen by the plan
    int force_cols = 0;      // tensor-core expansion tile width (32, 64, 128); 0: chosen by the plan
    int force_kstage = 0;    // K stage of its 128-column tiles (32, 64); 0: chosen by the plan
    int diag_basis = 6;      // Davidson basis limit, in blocks of b vectors
    int stall_iters = 10;    // learned-factor stall check: window and required fall (2^stall_log2)
    int stall_log2 = 1;
    int c4_path = 0;         // mixed class 4: 0 tensor cores for 32..64 states, 1 double-float only, 2 tensor cores for 1..64
    int64_t Pt = 0;
    int K = 0, Kpad = 0;
    // expansion panel columns: without orbital symmetry every label (n_cls 1,
    // Kc = Kpad); with it, 8 label classes (the irrep of the label's target
    // pair; h and delta in class 0) and Kc columns per class, padded to 64
    int n_cls = 1, Kc = 0;
    int32_t *cls_labels = nullptr;          // device [n_cls][Kc]: the labels of each class (-1 padding)
    std::vector<int32_t> cls_labels_h;
    std::vector<int32_t> co_irrep;          // irrep of every continuum orbital (empty without symmetry)
    int32_t *co_irrep_d = nullptr;
    int delta_pos = 0;                      // panel column of the delta label (in class 0)
    // the panel column list of the rectangle whose first continuum orbitals
    // are cf and cfp (null without symmetry)
    int class_of(int cf, int cfp) const {
        const int n = (int)co_irrep.size();
        return (n_cls > 1 && cf >= 0 && cf < n && cfp >= 0 && cfp < n) ? (co_irrep[cf] ^ co_irrep[cfp]) : 0;
    }
    const int32_t *class_labels(int cf, int cfp) const {
        return n_cls > 1 ? cls_labels + (int64_t)class_of(cf, cfp) * Kc : nullptr;
    }
    int64_t Dc = 0, dim = 0;
    std::vector<hb::GroupInfo> groups;
    std::vector<hb::GroupPair> gps;
    std::vector<hb::GroupL2> gl2;
    std::vector<void *> allocs;
    size_t dev_bytes = 0;
    double *h = nullptr, *tttt = nullptr, *tttc = nullptr, *jk = nullptr, *panel = nullptr;
    uint64_t *dets = nullptr, *l2 = nullptr;
    double *ci = nullptr;
    // target-energy substitution (Section 3.1): every group's state energies,
    // or null when the target-only part is the Eq. 8 sum
    double *energy = nullptr;
    // first row of each input group when groups were merged (empty otherwise)
    std::vector<int64_t> user_row_off;
    // double-float (hi, lo) copies for the mixed class-4 kernel, made on first use
    float2 *tttc_df = nullptr, *h_df = nullptr, *ci_df = nullptr, *tttt_df = nullptr, *jk_df = nullptr;
    int64_t *l2_rowptr = nullptr;
    int32_t *l2_seg_off = nullptr;
    int64_t l2_nnz = 0, tt_pairs = 0, tl2_pairs = 0;
    // the L2 x L2 entries below the diagonal and their mirrors (null: none found)
    int64_t *l2_low_ptr = nullptr, *l2_mdst = nullptr, *l2_msrc = nullptr;
    int32_t *l2_mcol = nullptr;
    int64_t l2_nlow = 0;
    hb::MixedState *mixed = nullptr;
    hb::DevPool pool;        // device memory beyond the staged problem
    hb_ctx *base = nullptr;  // context whose staged integrals this one borrows (or null)
    void *plan = nullptr;    // cached grouped-launch plan of this context's own builds (k_plan.cu)
    void *shard_plan = nullptr;   // cached plan of this context's share of a sharded build
    void *diag = nullptr;   // Davidson workspace (k_davidson.cu)
    void *mlp = nullptr;    // learned preconditioner weights (k_mlp.cu)
    void *c4tc = nullptr;   // class-4 tensor-core operands (k_class4_tc.cu)

    hb::Ints ints() const {
        hb::Ints I;
        I.h = h; I.tttt = tttt; I.tttc = tttc; I.jk = jk;
        I.h_df = h_df; I.tttt_df = tttt_df; I.jk_df = jk_df;
        I.n_to = n_to; I.n_co = n_co; I.n_orb = n_orb; I.Pt = Pt;
        return I;
    }
};

int stage_problem(hb_ctx *ctx, const hb_problem *p, const hb_options *o, cudaStream_t s);
void release_mixed(hb_ctx *ctx);
// Make the double-float copies of (tt|tc), h and the CI vectors (borrowing the
// integrals' copies from the base context).
int ensure_df(hb_ctx *ctx, cudaStream_t s);
