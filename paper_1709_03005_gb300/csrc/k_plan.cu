// Build plan: the whole build of one or many staged Hamiltonians as a short,
// fixed sequence of grouped launches.
//
// Every stage of the path (K1 classification, the H^N values, the S / E
// sandwiches, the gamma items, their counting sort and bins, the coefficient
// rows, the Eq. 7 expansion, class 4, the L2 CSR) is launched once for all
// target-group pairs (or groups, or L2 sets) of all Hamiltonians of the plan:
// each task owns a block range of the grid (hb_tasks.cuh), so uneven blocks
// of different size share the GPU within one launch instead of queueing as
// thousands of small launches.  The task tables live in one device buffer,
// uploaded when the plan is made (and again only when the output blocks
// change).  A plan over many contexts is what a batch captures in a CUDA graph.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include "hb_c4tc.cuh"
#include "hb_plan.cuh"
#include "hb_split.cuh"
#include "hb_tasks.cuh"

namespace hb {

template <class T>
struct Stage {
    std::vector<T> tasks;
    std::vector<int64_t> blk{0};
    size_t off_t = 0, off_b = 0;
    Grouped<T> g;
    void add(const T &t, int64_t blocks) {
        tasks.push_back(t);
        blk.push_back(blk.back() + (blocks > 0 ? blocks : 0));
    }
    void clear() {
        tasks.clear();
        blk.assign(1, 0);
    }
};

// Labels of the class of the rectangle whose first continuum orbitals are cf,
// cfp (every label without orbital symmetry): the K of its Eq. 7 sums.
static int class_label_count(const hb_ctx *ctx, int cf, int cfp) {
    if (ctx->n_cls <= 1) return ctx->K;
    const int x = ctx->class_of(cf, cfp);
    int c = 0;
    for (int i = 0; i < ctx->Kc; ++i) c += ctx->cls_labels_h[(size_t)x * ctx->Kc + i] >= 0;
    return c;
}

struct SplitGroup {
    const hb_ctx *panel_ctx = nullptr;
    int lg = 4;                        // tile arrangement of every task of the launch
    int bn = 128;                      // tile width (columns) of every task of the launch
    Stage<SplitTask> st;
};

// Tunable launch shapes.  Every candidate of a choice computes bit-identical
// results (only the partition of the work over blocks and threads changes),
// so tuning never changes the output.
struct Choices {
    std::map<std::pair<int, int>, int> tile;                   // (cn, cn') -> split tile arrangement
    std::map<std::pair<int, int>, std::pair<int, int>> c4;     // (ns, cn) -> (state tile, threads)
    std::map<int, int> gamma_warp;                             // ns * ns' (<= 64) -> 1 warp / 0 block per key
};

// What the tuner needs of each tunable task.
struct TuneSplit {
    const hb_ctx *panel_ctx;
    SplitTask t;
};
struct TuneC4 {
    C4Task t;
};
struct TuneGamma {
    GTask t;
};

struct Plan {
    std::vector<hb_ctx *> ctxs;
    std::vector<hb_blocks> outs;
    int precision = HB_FP64;
    int W = 1, Kpad = 0, n_to = 0, S = 0, delta_col = 0;
    // panel columns per label class (Kc) and the coefficient slices' width
    // (Kw = every class); perm: the labels of the coefficient slice columns
    // (null without orbital symmetry)
    int Kc = 0, Kw = 0;
    const int32_t *perm = nullptr;
    Stage<ClsTask> cls_tt, cls_tl2;
    Stage<PVTask> pv;
    Stage<PVTask> pvd;                 // the diagonal records of same-group pairs
    Stage<SWTask> sw, sws;             // sandwich: lanes over records / over states
    int sw_width = 16;                 // states per pass of the record-lane sandwich
    Stage<TNTask> tn, tnr;
    Stage<IFTask> itf;
    Stage<ZTask> zero;
    Stage<SortTask> sort;
    Stage<ScanTask> scan;
    Stage<GTask> gam, gamw;            // gamma bins: block / warp (ns * nsp <= 64) per key
    Stage<GDTask> gdp, gdr;            // diagonal gamma of same-group pairs: partial sums, reduction
    size_t smem_gd = 0;
    Stage<ATask> asmb;
    Stage<XTask> x64;
    Stage<SliceTask> slc;
    std::vector<SplitGroup> split;
    Stage<DRTask> drows;
    struct C4Var {
        int ns_tile, jt;
        Stage<C4Task> st;
    };
    std::vector<C4Var> c4v;            // class-4 launch shapes (one grouped launch each)
    Stage<C4FTask> c4f;                // class 4 on the tensor cores: term lists, then the GEMMs
    Stage<C4TTask> c4t;
    Stage<L2Task> l2;
    Stage<L2MTask> l2m;          // the L2 x L2 entries below the diagonal, after l2
    std::vector<ExpCol> cols;          // columns of the merged expansion blocks
    size_t off_cols = 0;
    const ExpCol *d_cols = nullptr;
    std::vector<C4Item> c4items;       // work items of the tensor-core class-4 launch
    size_t off_c4items = 0;
    const C4Item *d_c4items = nullptr;
    size_t smem_tn = 0, smem_gamma = 0;
    double flops = 0.0;
    int n_expand_tasks = 0;
    // device copies of the task tables
    std::vector<uint8_t> host;
    uint8_t *dev = nullptr, *pinned = nullptr;
    size_t dev_size = 0;
    cudaEvent_t uploaded = nullptr;
    bool upload_pending = false;
    // tensor-core operands
    void *coef = nullptr;
    CUtensorMap tm_coef[4];            // coefficient slices: 32-K stages at widths 32, 64, 128; 64-K at 128
    int64_t coef_rows = 0;
    int *err = nullptr;
    // classes 4, 2 and 8 run on a second stream beside the target side and
    // the expansion (they read only staged data and write their own blocks);
    // the target side and the expansion at higher priority, the second stream
    // taking the SMs they leave
    cudaStream_t main = nullptr, side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, join_main = nullptr;
    // the target side's independent chains: the diagonal H^N values and the
    // gamma items (aux1), the diagonal gamma (aux2), beside the E, S chain
    cudaStream_t aux1 = nullptr, aux2 = nullptr;
    cudaEvent_t k1_done = nullptr, items_done = nullptr, gd_done = nullptr, dv_done = nullptr;
    cudaEvent_t c4_done = nullptr;     // the tensor-core class-4 kernel has finished (side stream)
    // timers: start, target, expansion (main stream); class-4 end, L2 end, side
    // start (side stream); end after the join; L2 start, class-4 classification
    // end (side stream); split kernels
    cudaEvent_t ev[9] = {};
    std::vector<cudaEvent_t> ev_split;
    int launches = 0, expand_launches = 0;
    bool timed = false;
    Choices choice;
    bool tuned = false;
    std::vector<TuneSplit> tune_split;
    std::vector<TuneC4> tune_c4;
    std::vector<TuneGamma> tune_gamma;
    // sharded build (Section 3.1): rank shard_r of shard_n takes the bra
    // determinants [ndet r / n, ndet (r + 1) / n) of every group pair in the
    // prototype contraction, every shard_n-th expansion tile from shard_r, and
    // the L2 rows [n_l2 r / n, n_l2 (r + 1) / n) of classes 4, 2 and 8.
    // phase 1 runs the contraction only, phase 2 the rest, 0 everything.
    int shard_r = 0, shard_n = 1, phase = 0;
    std::vector<std::pair<int64_t, int64_t>> item_range;   // per group pair of ctxs[0]: its rows' gamma items
};

// First and last-plus-one of n items that rank r of R takes.
inline std::pair<int64_t, int64_t> shard_range(int64_t n, int r, int R) {
    return {n * r / R, n * (r + 1) / R};
}

}  // namespace hb

using namespace hb;

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <class T>
void stage_pack(Stage<T> &st, std::vector<uint8_t> &host) {
    st.off_t = align256(host.size());
    host.resize(st.off_t + sizeof(T) * st.tasks.size());
    if (!st.tasks.empty()) memcpy(host.data() + st.off_t, st.tasks.data(), sizeof(T) * st.tasks.size());
    st.off_b = align256(host.size());
    host.resize(st.off_b + sizeof(int64_t) * st.blk.size());
    memcpy(host.data() + st.off_b, st.blk.data(), sizeof(int64_t) * st.blk.size());
}

template <class T>
void stage_bind(Stage<T> &st, uint8_t *dev) {
    st.g.tasks = (const T *)(dev + st.off_t);
    st.g.blk = (const int64_t *)(dev + st.off_b);
    st.g.n = (int)st.tasks.size();
    st.g.blocks = st.blk.back();
}

// Task tables of every stage from the contexts and the output blocks.
void fill_tasks(Plan &p) {
    p.cls_tt.clear(); p.cls_tl2.clear(); p.pv.clear(); p.pvd.clear(); p.sw.clear(); p.sws.clear(); p.sw_width = 16; p.gamw.clear(); p.gdp.clear(); p.gdr.clear(); p.tn.clear(); p.tnr.clear();
    p.itf.clear(); p.zero.clear(); p.sort.clear(); p.scan.clear(); p.gam.clear(); p.asmb.clear();
    p.x64.clear(); p.slc.clear(); p.drows.clear(); p.l2.clear(); p.l2m.clear();
    for (auto &v : p.c4v) v.st.clear();
    p.c4f.clear(); p.c4t.clear();
    for (auto &sg : p.split) sg.st.clear();
    p.cols.clear();
    p.c4items.clear();
    p.tune_split.clear(); p.tune_c4.clear(); p.tune_gamma.clear();
    p.smem_tn = p.smem_gamma = p.smem_gd = 0;
    p.flops = 0.0;
    p.n_expand_tasks = 0;
    int64_t coef_row = 0;
    // expansion blocks: the group pairs (of any context) that read the same
    // continuum rectangle of the same panel share one GEMM
    struct BlockKey {
        const void *panel;
        int cf, cn, cfp, cnp;
        bool operator<(const BlockKey &o) const {
            if (panel != o.panel) return panel < o.panel;
            if (cf != o.cf) return cf < o.cf;
            if (cn != o.cn) return cn < o.cn;
            if (cfp != o.cfp) return cfp < o.cfp;
            return cnp < o.cnp;
        }
    };
    struct Member {
        hb_ctx *ctx;
        const GroupPair *P;
        const hb_blocks *out;
    };
    struct Block {
        BlockKey key;
        hb_ctx *ctx = nullptr;
        std::vector<Member> members;
    };
    std::map<BlockKey, int> block_of;
    std::vector<Block> blocks;
    for (size_t ci = 0; ci < p.ctxs.size(); ++ci) {
        hb_ctx *ctx = p.ctxs[ci];
        const hb_blocks &out = p.outs[ci];
        const Ints I = ctx->ints();
        const int n_keys = 2 * ctx->n_to * ctx->n_to;
        const int W = ctx->W;
        for (auto &P : ctx->gps) {
            const GroupInfo &A = ctx->groups[P.g], &B = ctx->groups[P.gp];
            const uint64_t *da = ctx->dets + A.det_off, *db = ctx->dets + B.det_off;
            const double *Ca = ctx->ci + A.ci_off, *Cb = ctx->ci + B.ci_off;
            const float2 *Ca_df = ctx->ci_df ? ctx->ci_df + A.ci_off : nullptr;
            const float2 *Cb_df = ctx->ci_df ? ctx->ci_df + B.ci_off : nullptr;
            p.cls_tt.add(ClsTask{da, db, A.ndet, B.ndet, ctx->cont_spin, 2, 0, P.rowptr, P.seg_off, seg_count(B.ndet),
                                 P.pairs},
                         blocks_seg_rows8(A.ndet, B.ndet));
            const PVTask pvt{I, da, db, P.pairs, P.n_pairs, P.val, P.rowptr, A.ndet, P.same};
            p.pv.add(pvt, blocks_pair_values(P.n_pairs));
            if (P.same) p.pvd.add(pvt, blocks_diag_values(A.ndet));
            // the bra rows this rank contracts (all of them unless sharded)
            const auto mr = shard_range(A.ndet, p.shard_r, p.shard_n);
            const int m0 = (int)mr.first, nm = (int)(mr.second - mr.first);
            // lanes over the states for at most 16 of them (two or more record
            // groups per warp), lanes over the records otherwise
            {
                const SWTask sw{P.pairs, P.rowptr + m0, P.val, nm, Cb, Cb_df, B.ns, P.W + (int64_t)m0 * B.ns};
                if (B.ns <= 16) p.sws.add(sw, blocks_rows8(nm));
                else p.sw.add(sw, nm);                        // a block per row
            }
            if (B.ns > 16) p.sw_width = std::max(p.sw_width, B.ns <= 24 ? 24 : 32);
            const int ny = tn_ny(A.ns, B.ns);
            // E = C^T (H^N C'); S = C^T C within a group (identical determinants
            // only, hb_init rejects repeats) and zero between groups; over this
            // rank's bra rows
            const double *Cm = Ca + (int64_t)m0 * A.ns, *Wm = P.W + (int64_t)m0 * B.ns;
            const float2 *Cm_df = Ca_df ? Ca_df + (int64_t)m0 * A.ns : nullptr;
            const TNTask te{Cm, Wm, Cm_df, reinterpret_cast<const float2 *>(Wm), nm, A.ns, B.ns, ny, P.partial, P.E};
            const TNTask ts{Cm, Cm, Cm_df, Cm_df, P.same ? nm : 0, A.ns, B.ns, ny, P.partial_s, P.S};
            p.tn.add(te, blocks_tn_partial(te.n_rows, A.ns, B.ns));
            p.tn.add(ts, blocks_tn_partial(ts.n_rows, A.ns, B.ns));
            p.tnr.add(te, blocks_tn_reduce(A.ns, B.ns));
            p.tnr.add(ts, blocks_tn_reduce(A.ns, B.ns));
            p.smem_tn = std::max(p.smem_tn, smem_stage(A.ns, B.ns));
            // the gamma items of this rank's rows are the contiguous run
            // [item_ptr[m0], item_ptr[m1]) (items follow the records' order)
            int64_t i0 = 0, n_it = P.n_items;
            if (p.shard_n > 1) {
                const auto &ir = p.item_range[&P - ctx->gps.data()];
                i0 = ir.first;
                n_it = ir.second - ir.first;
            }
            p.itf.add(IFTask{P.pairs, P.rowptr + m0, nm, da, W, ctx->n_to, ctx->n_elec, P.item_ptr + m0, P.items},
                      nm);                                    // a block per row
            const int nc = P.n_chunks;
            const int64_t n_off = (int64_t)n_keys * nc;
            GammaItem *its = P.items + i0;
            p.zero.add(ZTask{P.sort_off, n_off + 1}, blocks_zero(n_off + 1));
            p.sort.add(SortTask{its, n_it, nc, n_keys, P.sort_off, P.sort_cur, P.order}, blocks_sort(n_it, n_keys));
            p.scan.add(ScanTask{P.sort_off, n_off, P.sort_cur, P.sort_part}, blocks_scan(n_off));
            const GTask gt{its, P.order, P.sort_off, nc, n_keys, Ca, Ca_df, A.ns, Cb, Cb_df, B.ns, ny, P.gamma};
            const int nout = A.ns * B.ns;
            bool warp = nout <= 64;
            if (warp) {
                auto gc = p.choice.gamma_warp.find(nout);
                if (gc != p.choice.gamma_warp.end()) warp = gc->second != 0;
                p.tune_gamma.push_back(TuneGamma{gt});
            }
            if (warp) {
                p.gamw.add(gt, blocks_gamma_warp(n_keys));
            } else {
                p.gam.add(gt, blocks_gamma(n_keys, A.ns, B.ns));
                p.smem_gamma = std::max(p.smem_gamma, smem_stage(A.ns, B.ns));
            }
            if (P.same) {
                const GDTask gd{da + (int64_t)m0 * 2 * W, W, ctx->n_to, nm, A.ns, tn_ny(A.ns, A.ns), Cm, Cm_df,
                                P.gdiag, P.gamma};
                p.gdp.add(gd, blocks_gdiag_partial(nm, ctx->n_to, A.ns));
                p.gdr.add(gd, blocks_gdiag_reduce(ctx->n_to, A.ns));
                p.smem_gd = std::max(p.smem_gd, smem_gdiag(A.ns));
            }
            // with the target-energy substitution the energies are added once, by rank 0
            p.asmb.add(ATask{P.gamma, P.S, P.E, P.sort_off, nc, P.same, P.nn, P.n_nn, A.ns, B.ns, ctx->n_to,
                             ctx->cont_spin, ctx->Kpad,
                             ctx->e_core, P.A, p.precision == HB_MIXED ? P.A_df : nullptr,
                             ctx->energy ? ctx->energy + A.e_off : nullptr, ctx->energy && p.shard_r != 0},
                       P.n_nn);
            p.flops += 2.0 * (double)A.cn * B.cn * P.n_nn * class_label_count(ctx, A.cf, B.cf);
            ++p.n_expand_tasks;
            // the pair joins the expansion block of its continuum rectangle
            const BlockKey key{(const void *)ctx->panel, A.cf, A.cn, B.cf, B.cn};
            auto it = block_of.find(key);
            if (it == block_of.end()) {
                it = block_of.emplace(key, (int)blocks.size()).first;
                blocks.emplace_back();
                blocks.back().key = key;
                blocks.back().ctx = ctx;
            }
            blocks[it->second].members.push_back(Member{ctx, &P, &out});
            if (p.precision == HB_MIXED && p.shard_r == 0) {     // the j == j' rows: the first shard
                const int j_lo = std::max(A.cf, B.cf), j_hi = std::min(A.cf + A.cn, B.cf + B.cn);
                // rows j == j' are of class 0 (irrep(j) ^ irrep(j) = 0)
                p.drows.add(DRTask{mixed_panel_diag(ctx), P.A_df, P.nn, ctx->n_cls > 1 ? ctx->cls_labels : nullptr,
                                   P.n_nn, ctx->Kc, ctx->Kpad, ctx->n_co, j_lo, j_hi, A.cf, A.cn,
                                   B.cf, B.cn, P.same, diag_rows_ny(P.n_nn), A.row_off, B.row_off, ctx->Dc, out.Hcc},
                            blocks_diag_rows(j_lo, j_hi, P.n_nn));
            }
        }
        // the L2 rows of classes 4, 2 and 8 this rank builds
        const auto lr = shard_range(ctx->n_l2, p.shard_r, p.shard_n);
        const int l0 = (int)lr.first, nl = (int)(lr.second - lr.first);
        for (int g = 0; g < ctx->n_groups; ++g) {
            const GroupInfo &G = ctx->groups[g];
            GroupL2 &L = ctx->gl2[g];
            const uint64_t *dg = ctx->dets + G.det_off;
            p.cls_tl2.add(ClsTask{ctx->l2, dg, ctx->n_l2, G.ndet, ctx->cont_spin, 2, 0, L.rowptr, L.seg_off,
                                  seg_count(G.ndet), L.pairs},
                          blocks_seg_rows8(ctx->n_l2, G.ndet));
            if (p.precision == HB_MIXED && c4tc_group_on(ctx, g)) {
                C4FTask ft;
                C4TTask tt;
                int64_t fb = 0, items = 0;
                c4tc_tasks(ctx, g, out.Hlc, &ft, &fb, &tt, &items);
                const size_t first = p.c4items.size();
                c4tc_items(ctx, g, (int)p.c4t.tasks.size(), &p.c4items);
                if (p.shard_n > 1) {
                    // this rank's L2 rows only
                    auto keep = std::remove_if(p.c4items.begin() + first, p.c4items.end(), [&](const C4Item &c) {
                        return c.l < l0 || c.l >= l0 + nl;
                    });
                    p.c4items.erase(keep, p.c4items.end());
                    items = (int64_t)(p.c4items.size() - first);
                }
                p.c4f.add(ft, fb);
                p.c4t.add(tt, items);
                continue;
            }
            int ns_tile = 32, jt = 128;
            if (p.precision == HB_MIXED) {
                class4_shape(G.ns, G.cn, &ns_tile, &jt);
                auto cc = p.choice.c4.find({G.ns, G.cn});
                if (cc != p.choice.c4.end()) { ns_tile = cc->second.first; jt = cc->second.second; }
                if (ctx->force_c4_states) ns_tile = ctx->force_c4_states;
                if (ctx->force_c4_threads) jt = ctx->force_c4_threads;
            }
            Plan::C4Var *var = nullptr;
            for (auto &v : p.c4v)
                if (v.ns_tile == ns_tile && v.jt == jt) var = &v;
            if (!var) {
                p.c4v.push_back(Plan::C4Var{ns_tile, jt, Stage<C4Task>()});
                var = &p.c4v.back();
            }
            const C4Task c4t{I, L.pairs, L.rowptr + l0, nl, dg, ctx->ci + G.ci_off,
                             ctx->ci_df ? ctx->ci_df + G.ci_off : nullptr, ctx->tttc_df, ctx->h_df, G.ns, G.cf, G.cn,
                             ctx->cont_spin, class4_ny(G.cn, jt), G.row_off, ctx->Dc,
                             out.Hlc ? out.Hlc + (int64_t)l0 * ctx->Dc : nullptr};
            var->st.add(c4t, blocks_class4(nl, G.cn, jt));
            if (p.precision == HB_MIXED) p.tune_c4.push_back(TuneC4{c4t});
        }
        if (ctx->n_l2 > 0) {
            p.l2.add(L2Task{I, ctx->l2, ctx->n_l2, seg_count(ctx->n_l2), ctx->l2_rowptr, ctx->l2_seg_off, out.l2_row_ptr,
                            out.l2_col, out.l2_val, ctx->e_core, ctx->l2_low_ptr, l0, l0 + nl},
                     blocks_seg_rows8(ctx->n_l2, ctx->n_l2));
            // an entry below the diagonal is copied by the rank that evaluates its
            // mirror, whose row is the entry's column
            if (ctx->l2_low_ptr && ctx->l2_nlow > 0)
                p.l2m.add(L2MTask{ctx->l2_mdst, ctx->l2_msrc, ctx->l2_mcol, ctx->l2_nlow, out.l2_col, out.l2_val,
                                  l0, l0 + nl},
                          (ctx->l2_nlow + kL2MirrorThreads - 1) / kL2MirrorThreads);
        }
    }
    // merged expansion blocks: columns member by member, state pairs in order
    for (auto &B : blocks) {
        const int64_t col0 = (int64_t)p.cols.size();
        for (const Member &m : B.members) {
            const GroupPair &P = *m.P;
            const int64_t mstart = (int64_t)p.cols.size();
            const GroupInfo &A = m.ctx->groups[P.g], &Bg = m.ctx->groups[P.gp];
            int t = 0;
            for (int a = 0; a < A.ns; ++a)
                for (int b = 0; b < Bg.ns; ++b) {
                    if (P.same && b > a) continue;
                    ExpCol c;
                    c.arow = P.A + (int64_t)t * m.ctx->Kpad;
                    c.H = m.out->Hcc;
                    c.rbase = A.row_off + (int64_t)a * A.cn;
                    c.cbase = Bg.row_off + (int64_t)b * Bg.cn;
                    c.ld = m.ctx->Dc;
                    c.same = P.same;
                    c.pad = 0;
                    p.cols.push_back(c);
                    ++t;
                }
            if (p.precision == HB_MIXED)
                p.slc.add(SliceTask{P.A, P.n_nn, coef_row + (mstart - col0)}, P.n_nn);   // a block per row
        }
        const int N = (int)((int64_t)p.cols.size() - col0);
        const BlockKey &k = B.key;
        if (p.precision == HB_MIXED) {
            int lg = split_tile_heuristic(k.cn, k.cnp);
            auto tc = p.choice.tile.find({k.cn, k.cnp});
            if (tc != p.choice.tile.end()) lg = tc->second;
            if (B.ctx->force_tile) lg = B.ctx->force_tile;
            const int bn = split_cols_choice(N, p.Kc / 64, B.ctx->force_cols);
            const void *pkey = mixed_panel_key(B.ctx);
            int gi = -1;
            for (size_t i = 0; i < p.split.size(); ++i)
                if (mixed_panel_key(p.split[i].panel_ctx) == pkey && p.split[i].lg == lg && p.split[i].bn == bn)
                    gi = (int)i;
            if (gi < 0) {
                p.split.emplace_back();
                p.split.back().panel_ctx = B.ctx;
                p.split.back().lg = lg;
                p.split.back().bn = bn;
                gi = (int)p.split.size() - 1;
            }
            SplitTask t;
            t.cf = k.cf; t.cn = k.cn; t.cfp = k.cfp; t.cnp = k.cnp;
            t.bjp_log2 = lg;
            t.jpt_tiles = split_jpt(k.cnp, lg);
            t.bn = bn;
            t.ntn = split_ntn(N, bn);
            t.N = N;
            t.coef_row0 = coef_row;
            t.col0 = col0;
            t.kc0 = B.ctx->class_of(k.cf, k.cfp) * (p.Kc / 64);
            p.split[gi].st.add(t, blocks_split(k.cn, k.cnp, N, lg, bn));
            p.tune_split.push_back(TuneSplit{B.ctx, t});
            coef_row += N;
        } else {
            p.x64.add(XTask{B.ctx->panel, B.ctx->Kc, B.ctx->n_co, k.cf, k.cn, k.cfp, k.cnp,
                            expand_fp64_mtiles(k.cn, k.cnp), N, col0, B.ctx->class_labels(k.cf, k.cfp)},
                      blocks_expand_fp64(k.cn, k.cnp, N));
        }
    }
    p.coef_rows = coef_row;
}

void ensure_split_events(Plan &p) {
    while (p.ev_split.size() < 2 * p.split.size()) {
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        p.ev_split.push_back(e);
    }
}

void pack_all(Plan &p) {
    p.host.clear();
    stage_pack(p.cls_tt, p.host); stage_pack(p.cls_tl2, p.host); stage_pack(p.pv, p.host); stage_pack(p.pvd, p.host);
    stage_pack(p.sw, p.host); stage_pack(p.sws, p.host); stage_pack(p.gamw, p.host);
    stage_pack(p.gdp, p.host); stage_pack(p.gdr, p.host); stage_pack(p.tn, p.host); stage_pack(p.tnr, p.host); stage_pack(p.itf, p.host);
    stage_pack(p.zero, p.host); stage_pack(p.sort, p.host); stage_pack(p.scan, p.host); stage_pack(p.gam, p.host);
    stage_pack(p.asmb, p.host); stage_pack(p.x64, p.host); stage_pack(p.slc, p.host);
    for (auto &sg : p.split) stage_pack(sg.st, p.host);
    stage_pack(p.drows, p.host); stage_pack(p.l2, p.host); stage_pack(p.l2m, p.host);
    for (auto &v : p.c4v) stage_pack(v.st, p.host);
    stage_pack(p.c4f, p.host); stage_pack(p.c4t, p.host);
    p.off_cols = align256(p.host.size());
    p.host.resize(p.off_cols + sizeof(ExpCol) * p.cols.size());
    if (!p.cols.empty()) memcpy(p.host.data() + p.off_cols, p.cols.data(), sizeof(ExpCol) * p.cols.size());
    p.off_c4items = align256(p.host.size());
    p.host.resize(p.off_c4items + sizeof(C4Item) * p.c4items.size());
    if (!p.c4items.empty())
        memcpy(p.host.data() + p.off_c4items, p.c4items.data(), sizeof(C4Item) * p.c4items.size());
}

void bind_all(Plan &p) {
    stage_bind(p.cls_tt, p.dev); stage_bind(p.cls_tl2, p.dev); stage_bind(p.pv, p.dev); stage_bind(p.pvd, p.dev);
    stage_bind(p.sw, p.dev); stage_bind(p.sws, p.dev); stage_bind(p.gamw, p.dev);
    stage_bind(p.gdp, p.dev); stage_bind(p.gdr, p.dev); stage_bind(p.tn, p.dev); stage_bind(p.tnr, p.dev); stage_bind(p.itf, p.dev);
    stage_bind(p.zero, p.dev); stage_bind(p.sort, p.dev); stage_bind(p.scan, p.dev); stage_bind(p.gam, p.dev);
    stage_bind(p.asmb, p.dev); stage_bind(p.x64, p.dev); stage_bind(p.slc, p.dev);
    for (auto &sg : p.split) stage_bind(sg.st, p.dev);
    stage_bind(p.drows, p.dev); stage_bind(p.l2, p.dev); stage_bind(p.l2m, p.dev);
    for (auto &v : p.c4v) stage_bind(v.st, p.dev);
    stage_bind(p.c4f, p.dev); stage_bind(p.c4t, p.dev);
    p.d_cols = (const ExpCol *)(p.dev + p.off_cols);
    p.d_c4items = (const C4Item *)(p.dev + p.off_c4items);
}

// Copy the packed tables through the pinned staging buffer (which is reused
// only after the previous copy from it has finished).
int upload(Plan &p, std::string *err, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (p.upload_pending) e = cudaEventSynchronize(p.uploaded);
    p.upload_pending = false;
    if (e == cudaSuccess && p.host.size() > p.dev_size) {
        if (p.dev) dfree(p.ctxs[0], p.dev);
        if (p.pinned) cudaFreeHost(p.pinned);
        p.dev = nullptr;
        p.pinned = nullptr;
        p.dev_size = 0;
        e = dmalloc_n(p.ctxs[0], &p.dev, p.host.size());
        if (e == cudaSuccess) e = cudaMallocHost((void **)&p.pinned, p.host.size());
        if (e == cudaSuccess) p.dev_size = p.host.size();
    }
    if (e == cudaSuccess && !p.host.empty()) {
        memcpy(p.pinned, p.host.data(), p.host.size());
        e = cudaMemcpyAsync(p.dev, p.pinned, p.host.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(p.uploaded, s);
        if (e == cudaSuccess) p.upload_pending = true;
    }
    if (e != cudaSuccess) {
        *err = std::string("plan upload: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? HB_ERR_OOM : HB_ERR_CUDA;
    }
    bind_all(p);
    return HB_OK;
}

}  // namespace

int plan_create(hb_ctx *const *ctxs, int n, const hb_blocks *outs, int precision, Plan **out, std::string *err,
                cudaStream_t s, int shard_r, int shard_n) {
    *out = nullptr;
    if (n < 1) { *err = "empty plan"; return HB_ERR_INVALID_ARG; }
    Plan *p = new Plan();
    p->ctxs.assign(ctxs, ctxs + n);
    p->outs.assign(outs, outs + n);
    p->precision = precision;
    p->W = ctxs[0]->W;
    p->Kpad = ctxs[0]->Kpad;
    p->n_to = ctxs[0]->n_to;
    p->Kc = ctxs[0]->Kc;
    p->Kw = ctxs[0]->n_cls * ctxs[0]->Kc;
    p->perm = ctxs[0]->n_cls > 1 ? ctxs[0]->cls_labels : nullptr;
    for (int i = 1; i < n; ++i) {
        if (ctxs[i]->W != p->W || ctxs[i]->Kpad != p->Kpad || ctxs[i]->n_to != p->n_to) {
            delete p;
            *err = "contexts of one plan must share the target orbital space (n_words, n_to)";
            return HB_ERR_INVALID_ARG;
        }
        if (ctxs[i]->n_cls != ctxs[0]->n_cls || ctxs[i]->cls_labels_h != ctxs[0]->cls_labels_h) {
            delete p;
            *err = "contexts of one plan must share the orbital symmetry (orb_irrep of the target orbitals)";
            return HB_ERR_INVALID_ARG;
        }
    }
    int rc = HB_OK;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 9 && e == cudaSuccess; ++i) e = cudaEventCreate(&p->ev[i]);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->uploaded, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->join_main, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->c4_done, cudaEventDisableTiming);
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->main, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, least);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->aux1, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->aux2, cudaStreamNonBlocking, greatest);
    for (cudaEvent_t *ev : {&p->k1_done, &p->items_done, &p->gd_done, &p->dv_done})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = dmalloc_n(ctxs[0], &p->err, 2);   // split kernel, class-4 kernel
    if (e == cudaSuccess) e = cudaMemsetAsync(p->err, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) {
        *err = std::string("plan: ") + cudaGetErrorString(e);
        plan_destroy(p);
        return HB_ERR_CUDA;
    }
    bool any_pairs = false;
    for (int i = 0; i < n; ++i) any_pairs = any_pairs || !ctxs[i]->gps.empty();
    if (precision == HB_MIXED && any_pairs) {
        for (int i = 0; i < n && rc == HB_OK; ++i) {
            if (ctxs[i]->gps.empty()) continue;
            rc = mixed_prepare(ctxs[i], s);
            if (rc != HB_OK) { *err = ctxs[i]->err; break; }
            const int S = mixed_slices(ctxs[i]);
            if (p->S == 0) p->S = S;
            else if (S != p->S) { rc = HB_ERR_INVALID_ARG; *err = "contexts of one plan use different split_slices"; }
        }
        if (rc != HB_OK) { plan_destroy(p); return rc; }
        p->delta_col = ctxs[0]->delta_pos;   // the delta label's column (class 0 comes first)
    }
    if (precision == HB_MIXED && p->S == 0) p->S = mixed_slices(ctxs[0]);
    // class 4 on the tensor cores: integral and CI slices, term-list sizes
    if (precision == HB_MIXED)
        for (int i = 0; i < n && rc == HB_OK; ++i) {
            if (ctxs[i]->n_l2 < 1 || ctxs[i]->c4_path == 1) continue;
            rc = c4tc_prepare(ctxs[i], p->S, s);
            if (rc != HB_OK) *err = ctxs[i]->err;
        }
    if (precision == HB_MIXED)
        for (int i = 0; i < n && rc == HB_OK; ++i) {
            rc = ensure_df(ctxs[i], s);
            if (rc != HB_OK) *err = ctxs[i]->err;
        }
    if (rc != HB_OK) { plan_destroy(p); return rc; }
    if (shard_n > 1) {
        // a sharded plan serves one context; the gamma items of this rank's
        // bra rows, per group pair, from the staged item offsets
        p->shard_r = shard_r;
        p->shard_n = shard_n;
        for (auto &P : ctxs[0]->gps) {
            const auto mr = shard_range(ctxs[0]->groups[P.g].ndet, shard_r, shard_n);
            int64_t a = 0, b = 0;
            cudaError_t e2 = cudaMemcpy(&a, P.item_ptr + mr.first, sizeof(int64_t), cudaMemcpyDeviceToHost);
            if (e2 == cudaSuccess) e2 = cudaMemcpy(&b, P.item_ptr + mr.second, sizeof(int64_t), cudaMemcpyDeviceToHost);
            if (e2 != cudaSuccess) {
                *err = std::string("shard item ranges: ") + cudaGetErrorString(e2);
                plan_destroy(p);
                return HB_ERR_CUDA;
            }
            p->item_range.push_back({a, b});
        }
    }
    fill_tasks(*p);
    if (precision == HB_MIXED && p->coef_rows > 0) {
        rc = split_coef_alloc(ctxs[0], p->S, p->coef_rows, p->Kw, &p->coef, p->tm_coef, err);
        if (rc != HB_OK) { plan_destroy(p); return rc; }
        ensure_split_events(*p);
    }
    pack_all(*p);
    rc = upload(*p, err, s);
    if (rc != HB_OK) { plan_destroy(p); return rc; }
    *out = p;
    return HB_OK;
}

bool plan_outputs_equal(const Plan *p, const hb_blocks *outs) {
    for (size_t i = 0; i < p->outs.size(); ++i) {
        const hb_blocks &a = p->outs[i], &b = outs[i];
        if (a.Hcc != b.Hcc || a.Hlc != b.Hlc || a.l2_row_ptr != b.l2_row_ptr || a.l2_col != b.l2_col ||
            a.l2_val != b.l2_val)
            return false;
    }
    return true;
}

int plan_precision(const Plan *p) { return p->precision; }

int plan_set_outputs(Plan *p, const hb_blocks *outs, std::string *err, cudaStream_t s) {
    p->outs.assign(outs, outs + p->outs.size());
    fill_tasks(*p);
    ensure_split_events(*p);
    pack_all(*p);
    return upload(*p, err, s);
}

namespace {

// Mean time of `launch` over a private copy of the given tasks (one warm-up
// launch, then `reps` timed launches on stream s).
template <class T, class F>
float time_tasks(hb_ctx *mem, const std::vector<T> &tasks, const std::vector<int64_t> &nblocks, F launch,
                 cudaStream_t s, int reps = 2) {
    std::vector<int64_t> blk(1, 0);
    for (int64_t b : nblocks) blk.push_back(blk.back() + b);
    if (tasks.empty() || blk.back() == 0) return 0.0f;
    const size_t bt = sizeof(T) * tasks.size(), ob = align256(bt), total = ob + sizeof(int64_t) * blk.size();
    uint8_t *d = nullptr;
    if (dmalloc_n(mem, &d, total) != cudaSuccess) return 1e30f;
    cudaMemcpyAsync(d, tasks.data(), bt, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d + ob, blk.data(), sizeof(int64_t) * blk.size(), cudaMemcpyHostToDevice, s);
    Grouped<T> g;
    g.tasks = (const T *)d;
    g.blk = (const int64_t *)(d + ob);
    g.n = (int)tasks.size();
    g.blocks = blk.back();
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch(g);
    cudaEventRecord(a, s);
    for (int r = 0; r < reps; ++r) launch(g);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamSynchronize(s);
    dfree(mem, d);
    return ms / reps;
}

}  // namespace

// A candidate replaces the heuristic default only if it is this much faster
// (short launches time noisily; a stage's tasks also share the GPU when the
// whole plan runs, which a timing of one class alone does not see).
constexpr float kGain = 0.95f;

int plan_autotune(Plan *p, cudaStream_t s, std::string *err) {
    // one build makes every stage's inputs (records, coefficient rows and their
    // slices) current; the candidates then rerun single stages on them
    int rc = plan_run(p, s, false, false, nullptr, err);
    if (rc != HB_OK) return rc;
    if (cudaStreamSynchronize(s) != cudaSuccess) { *err = "autotune: build failed"; return HB_ERR_CUDA; }
    const int W = p->W;
    Choices ch;
    // split expansion: tile arrangement per continuum rectangle (and panel)
    {
        std::map<std::tuple<const void *, int, int>, std::vector<const TuneSplit *>> cls;
        for (auto &t : p->tune_split) cls[{mixed_panel_key(t.panel_ctx), t.t.cn, t.t.cnp}].push_back(&t);
        for (auto &kv : cls) {
            const int cn = std::get<1>(kv.first), cnp = std::get<2>(kv.first);
            const hb_ctx *pc = kv.second.front()->panel_ctx;
            // the least-padding arrangement stays unless another is clearly faster
            const int def_lg = split_tile_heuristic(cn, cnp);
            float best = 0.0f, def_ms = 0.0f;
            int best_lg = -1;
            for (int lg : {def_lg, 3, 4, 5}) {
                if (best_lg >= 0 && lg == def_lg) continue;
                // the rectangle's blocks, one launch per tile width as in the build
                float ms = 0.0f;
                for (int bn : {32, 64, 128}) {
                    std::vector<SplitTask> ts;
                    std::vector<int64_t> nb;
                    for (auto *t : kv.second) {
                        if (t->t.bn != bn) continue;
                        SplitTask u = t->t;
                        u.bjp_log2 = lg;
                        u.jpt_tiles = split_jpt(cnp, lg);
                        ts.push_back(u);
                        nb.push_back(blocks_split(cn, cnp, u.N, lg, bn));
                    }
                    if (ts.empty()) continue;
                    ms += time_tasks(p->ctxs[0], ts, nb, [&](const Grouped<SplitTask> &g) {
                        g_split(pc, lg, bn, p->tm_coef, g, p->Kc / 64, p->Kw / 64, p->d_cols, p->err, s);
                    }, s);
                }
                if (best_lg < 0) { best = def_ms = ms; best_lg = lg; }
                else if (ms < best && ms < kGain * def_ms) { best = ms; best_lg = lg; }
            }
            // a rectangle seen with several panels keeps the first panel's choice
            ch.tile.emplace(std::make_pair(cn, cnp), best_lg);
        }
    }
    // class 4: state tile and thread count per (states, continuum count)
    {
        std::map<std::pair<int, int>, std::vector<const TuneC4 *>> cls;
        for (auto &t : p->tune_c4) cls[{t.t.ns, t.t.cn}].push_back(&t);
        for (auto &kv : cls) {
            const int cn = kv.first.second;
            int dnt = 32, djt = 128;
            class4_shape(kv.first.first, cn, &dnt, &djt);
            float best = 0.0f, def_ms = 0.0f;
            std::pair<int, int> arg(-1, -1);
            std::vector<std::pair<int, int>> cand{{dnt, djt}};
            for (int nt : {4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 56, 64})
                for (int jt : {32, 64, 128})
                    if (nt != dnt || jt != djt) cand.push_back({nt, jt});
            for (auto &c : cand) {
                const int nt = c.first, jt = c.second;
                std::vector<C4Task> ts;
                std::vector<int64_t> nb;
                for (auto *t : kv.second) {
                    C4Task u = t->t;
                    u.ny = class4_ny(cn, jt);
                    ts.push_back(u);
                    nb.push_back(blocks_class4(u.n_l2, cn, jt));
                }
                const float ms = time_tasks(p->ctxs[0], ts, nb, [&](const Grouped<C4Task> &g) {
                    g_class4(g, W, 1, nt, jt, s);
                }, s);
                if (arg.first < 0) { best = def_ms = ms; arg = c; }
                else if (ms < best && ms < kGain * def_ms) { best = ms; arg = c; }
            }
            ch.c4[kv.first] = arg;
        }
    }
    // gamma bins of small state blocks: one warp or one block per key
    {
        std::map<int, std::vector<const TuneGamma *>> cls;
        for (auto &t : p->tune_gamma) cls[t.t.ns * t.t.nsp].push_back(&t);
        for (auto &kv : cls) {
            std::vector<GTask> ts;
            std::vector<int64_t> nbw, nbb;
            size_t smem = 0;
            for (auto *t : kv.second) {
                ts.push_back(t->t);
                nbw.push_back(blocks_gamma_warp(t->t.n_keys));
                nbb.push_back(blocks_gamma(t->t.n_keys, t->t.ns, t->t.nsp));
                smem = std::max(smem, smem_stage(t->t.ns, t->t.nsp));
            }
            const int DF = p->precision == HB_MIXED ? 1 : 0;
            const float mw = time_tasks(p->ctxs[0], ts, nbw, [&](const Grouped<GTask> &g) { g_gamma_warp(g, DF, s); }, s);
            const float mb = time_tasks(p->ctxs[0], ts, nbb, [&](const Grouped<GTask> &g) { g_gamma(g, smem, DF, s); }, s);
            ch.gamma_warp[kv.first] = mb < kGain * mw ? 0 : 1;     // the warp form unless clearly slower
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { *err = std::string("autotune: ") + cudaGetErrorString(e); return HB_ERR_CUDA; }
    p->choice = ch;
    p->tuned = true;
    fill_tasks(*p);
    ensure_split_events(*p);
    pack_all(*p);
    return upload(*p, err, s);
}

bool plan_tuned(const Plan *p) { return p->tuned; }

void plan_set_phase(Plan *p, int phase) { p->phase = phase; }
bool plan_is_shard(const Plan *p, int precision, int r, int n) {
    return p->precision == precision && p->shard_r == r && p->shard_n == n;
}

std::string plan_report(const Plan *p) {
    std::string r;
    char buf[160];
    snprintf(buf, sizeof buf, "tuned=%d;", p->tuned ? 1 : 0);
    r += buf;
    std::map<std::pair<int, int>, int> tile;
    for (auto &g : p->split)
        for (auto &t : g.st.tasks) tile[{t.cn, t.cnp}] = g.lg;
    for (auto &kv : tile) {
        snprintf(buf, sizeof buf, " split %dx%d:%dx%d;", kv.first.first, kv.first.second, 128 >> kv.second,
                 1 << kv.second);
        r += buf;
    }
    for (auto &v : p->c4v)
        for (auto &t : v.st.tasks) {
            snprintf(buf, sizeof buf, " class4 ns%d cn%d:%dx%d;", t.ns, t.cn, v.ns_tile, v.jt);
            if (r.find(buf) == std::string::npos) r += buf;
        }
    if (!p->c4t.tasks.empty()) {
        snprintf(buf, sizeof buf, " class4 tensor cores: %d groups, %d work items;", (int)p->c4t.tasks.size(),
                 (int)p->c4items.size());
        r += buf;
    }
    snprintf(buf, sizeof buf, " gamma warp/block tasks %d/%d", (int)p->gamw.tasks.size(), (int)p->gam.tasks.size());
    r += buf;
    return r;
}

int plan_run(Plan *p, cudaStream_t s, bool timing, bool capture, int *launches, std::string *err) {
    int L = 0, LX = 0;
    const cudaStream_t s0 = s;
    const int W = p->W;
    // the mixed build runs the target side and class 4 in double-float on the
    // FP32 pipes, the plain build in FP64
    const int DF = p->precision == HB_MIXED ? 1 : 0;
    p->timed = timing;
    // inside a capture an event record becomes a graph node only when external
    auto rec_on = [&](cudaEvent_t e, cudaStream_t st) {
        if (!timing) return;
        if (capture) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
        else cudaEventRecord(e, st);
    };
    rec_on(p->ev[0], s);
    // fork: both chains wait for the caller's stream (inside a capture the
    // internal streams join the capture here)
    cudaStream_t s2 = p->side;
    cudaEventRecord(p->fork, s);
    cudaStreamWaitEvent(p->main, p->fork, 0);
    cudaStreamWaitEvent(s2, p->fork, 0);
    // class 4 (Eq. 5) and classes 2 and 8
    // the L2 rows stay FP64: their sums are short and the kernel is bound by the
    // pair scan, where the longer double-float sums cost more than FP64 adds
    rec_on(p->ev[5], s2);
    // a sharded build runs in two phases: the contraction (1), then, with the
    // reduced coefficient rows in place, classes 4, 2, 8 and the expansion (2)
    const bool ph1 = p->phase != 2, ph2 = p->phase != 1;
    if (ph2) L += g_classify(p->cls_tl2.g, W, 1, s2);
    rec_on(p->ev[8], s2);
    if (!ph2) {
        rec_on(p->ev[7], s2);
        rec_on(p->ev[4], s2);
        rec_on(p->ev[3], s2);
    } else if (p->c4t.g.blocks > 0) {
        // the tensor-core class-4 kernel and the expansion kernel each hold
        // whole SMs until their work is done, and the L2 rows' blocks do not
        // fit beside either: the L2 rows run beside the target side, then
        // class 4, and the expansion starts once both are done
        rec_on(p->ev[7], s2);
        L += g_l2_csr(p->l2.g, W, 0, s2);
        L += g_l2_mirror(p->l2m.g, s2);
        rec_on(p->ev[4], s2);
        cudaMemsetAsync(p->err + 1, 0, sizeof(int), s2);
        L += g_c4fill(p->c4f.g, s2);
        L += g_c4tc(p->c4t.g, p->d_c4items, (int)p->c4items.size(), p->S, p->err + 1, s2);
        for (auto &v : p->c4v) L += g_class4(v.st.g, W, 1, v.ns_tile, v.jt, s2);
        rec_on(p->ev[3], s2);
        cudaEventRecord(p->c4_done, s2);
    } else {
        for (auto &v : p->c4v) L += g_class4(v.st.g, W, p->precision == HB_MIXED ? 1 : 0, v.ns_tile, v.jt, s2);
        rec_on(p->ev[3], s2);
        rec_on(p->ev[7], s2);
        L += g_l2_csr(p->l2.g, W, 0, s2);
        L += g_l2_mirror(p->l2m.g, s2);
        rec_on(p->ev[4], s2);
    }
    cudaEventRecord(p->join, s2);
    s = p->main;
    auto rec = [&](cudaEvent_t e) { rec_on(e, s); };
    cudaStream_t sa = p->aux1, sb = p->aux2;
    // target side (Eq. 8) in three chains that meet at the coefficient rows:
    // the diagonal gamma needs only the determinants and CI vectors
    cudaStreamWaitEvent(sb, p->fork, 0);
    if (ph1) {
        L += g_gdiag(p->gdp.g, p->gdr.g, p->smem_gd, DF, sb);
        cudaEventRecord(p->gd_done, sb);
        L += g_classify(p->cls_tt.g, W, 0, s);
        cudaEventRecord(p->k1_done, s);
        // the gamma items of the single-excitation records, sorted by key, and gamma
        cudaStreamWaitEvent(sa, p->k1_done, 0);
        // the diagonal H^N values (a sequential sum per row) beside the others
        L += g_diag_values(p->pvd.g, W, DF, sa);
        cudaEventRecord(p->dv_done, sa);
        L += g_item_fill(p->itf.g, sa);
        L += g_zero(p->zero.g, sa);
        L += g_sort_hist(p->sort.g, sa);
        L += g_scan(p->scan.g, sa);
        L += g_sort_scatter(p->sort.g, sa);
        L += g_gamma(p->gam.g, p->smem_gamma, DF, sa);
        L += g_gamma_warp(p->gamw.g, DF, sa);
        cudaEventRecord(p->items_done, sa);
        // H^N values, the sandwich and E, S
        L += g_pair_values(p->pv.g, W, DF, s);
        cudaStreamWaitEvent(s, p->dv_done, 0);
        L += g_sandwich(p->sw.g, DF, p->sw_width, s);
        L += g_sandwich_small(p->sws.g, DF, s);
        L += g_tn_partial(p->tn.g, p->smem_tn, DF, s);
        L += g_tn_reduce(p->tnr.g, DF, s);
        cudaStreamWaitEvent(s, p->items_done, 0);
        cudaStreamWaitEvent(s, p->gd_done, 0);
        L += g_assemble(p->asmb.g, DF, s);
    } else {
        cudaEventRecord(p->gd_done, sb);   // the auxiliary stream joins the capture
        cudaStreamWaitEvent(s, p->gd_done, 0);
    }
    rec(p->ev[1]);
    // expansion (Eq. 7): classes 1, 3, 5, 6, 7
    if (!ph2) {
        // phase 1 ends with the coefficient rows
    } else if (p->precision == HB_MIXED) {
        // with class 4 on the tensor cores, the expansion waits for it (see
        // the side stream above); the double-float class-4 kernel runs beside
        // the expansion, which was faster than running it first
        if (p->c4t.g.blocks > 0) cudaStreamWaitEvent(s, p->c4_done, 0);
        if (p->coef_rows > 0) {
            cudaMemsetAsync(p->err, 0, sizeof(int), s);
            L += g_slice(p->slc.g, p->coef_rows, p->Kpad, p->Kw, p->perm, p->S, p->delta_col, p->coef, s);
            for (size_t i = 0; i < p->split.size(); ++i) {
                rec(p->ev_split[2 * i]);
                LX += g_split(p->split[i].panel_ctx, p->split[i].lg, p->split[i].bn, p->tm_coef, p->split[i].st.g, p->Kc / 64, p->Kw / 64,
                              p->d_cols, p->err, s,
                              p->shard_r, p->shard_n);
                rec(p->ev_split[2 * i + 1]);
            }
            // the rows with j == j' (double-float); beside the split kernel they
            // slowed it by more than they saved
            L += g_diag_rows(p->drows.g, s);
        }
    } else {
        LX += g_expand_fp64(p->x64.g, p->d_cols, s, p->shard_r, p->shard_n);
    }
    L += LX;
    rec(p->ev[2]);
    cudaEventRecord(p->join_main, s);
    // join into the caller's stream
    s = s0;
    cudaStreamWaitEvent(s, p->join_main, 0);
    cudaStreamWaitEvent(s, p->join, 0);
    rec(p->ev[6]);
    cudaError_t e = cudaGetLastError();
    p->launches = L;
    p->expand_launches = LX;
    if (launches) *launches = L;
    if (e != cudaSuccess) {
        *err = std::string("build launch: ") + cudaGetErrorString(e);
        return HB_ERR_CUDA;
    }
    return HB_OK;
}

void plan_stats(Plan *p, hb_stats *st) {
    memset(st, 0, sizeof(*st));
    st->kernel_launches = p->launches;
    st->expand_launches = p->expand_launches;
    st->expand_flops = p->flops;
    if (!p->timed) return;
    cudaEventSynchronize(p->ev[6]);
    cudaEventElapsedTime(&st->ms_total, p->ev[0], p->ev[6]);
    cudaEventElapsedTime(&st->ms_target, p->ev[0], p->ev[1]);
    cudaEventElapsedTime(&st->ms_expand, p->ev[1], p->ev[2]);
    cudaEventElapsedTime(&st->ms_l2, p->ev[7], p->ev[4]);
    if (p->c4t.g.blocks > 0) {
        // class-4 classification, then (after the L2 rows) the tensor-core part
        float a = 0.0f, b = 0.0f;
        cudaEventElapsedTime(&a, p->ev[5], p->ev[7]);
        cudaEventElapsedTime(&b, p->ev[4], p->ev[3]);
        st->ms_class4 = a + b;
        st->ms_class4_kernel = b;
    } else {
        cudaEventElapsedTime(&st->ms_class4, p->ev[5], p->ev[3]);
        cudaEventElapsedTime(&st->ms_class4_kernel, p->ev[8], p->ev[3]);
    }
    if (p->precision == HB_MIXED) {
        float total = 0.0f;
        for (size_t i = 0; i + 1 < p->ev_split.size(); i += 2) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, p->ev_split[i], p->ev_split[i + 1]) == cudaSuccess) total += t;
        }
        st->ms_expand_gemm = total;
        st->expand_tensor_flops = p->flops * (double)(p->S * (p->S + 1) / 2);
    } else {
        st->ms_expand_gemm = st->ms_expand;
    }
}

int plan_error_word(Plan *p, int *word) {
    *word = 0;
    if (!p->err) return HB_OK;
    int w[2] = {0, 0};
    if (cudaMemcpy(w, p->err, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return HB_ERR_CUDA;
    *word = w[0] ? w[0] : w[1];
    return HB_OK;
}

void plan_destroy(Plan *p) {
    if (!p) return;
    if (p->upload_pending) cudaEventSynchronize(p->uploaded);
    for (cudaEvent_t e : p->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : p->ev_split)
        if (e) cudaEventDestroy(e);
    if (p->uploaded) cudaEventDestroy(p->uploaded);
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->join) cudaEventDestroy(p->join);
    if (p->join_main) cudaEventDestroy(p->join_main);
    if (p->c4_done) cudaEventDestroy(p->c4_done);
    for (cudaEvent_t ev : {p->k1_done, p->items_done, p->gd_done, p->dv_done})
        if (ev) cudaEventDestroy(ev);
    for (cudaStream_t st : {p->main, p->side, p->aux1, p->aux2})
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    hb_ctx *mem = p->ctxs.empty() ? nullptr : p->ctxs[0];
    if (mem) {
        dfree(mem, p->dev);
        dfree(mem, p->coef);
        dfree(mem, p->err);
    }
    if (p->pinned) cudaFreeHost(p->pinned);
    delete p;
}

// Test hook (host only, not part of the interface): the tile width and K stage
// the plan gives a merged block of n_cols columns over kblocks 64-wide K blocks.
extern "C" int hb_test_split_shape(int n_cols, int kblocks, int force_cols, int force_kstage, int *cols,
                                   int *kstage) {
    if (!cols || !kstage || n_cols < 1 || kblocks < 1) return HB_ERR_INVALID_ARG;
    *cols = split_cols_choice(n_cols, kblocks, force_cols);
    *kstage = split_kstage_choice(*cols, kblocks, force_kstage);
    return HB_OK;
}
