// C ABI of the Hamiltonian build: validation, staging, orchestration.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_set>
#include <vector>

#include "hb_api_internal.cuh"
#include "hb_davidson.cuh"
#include "hb_c4tc.cuh"
#include "hb_plan.cuh"
#include "hb_df.cuh"
#include "hb_tasks.cuh"

using namespace hb;

namespace hb {
thread_local std::string g_last_error;
}

namespace {
int fail(hb_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    g_last_error = msg;
    return code;
}

int cuda_fail(hb_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? HB_ERR_OOM : HB_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

struct DetHash {
    size_t operator()(const std::vector<uint64_t> &v) const {
        uint64_t x = 0x9e3779b97f4a7c15ull;
        for (uint64_t w : v) x = (x ^ w) * 0xff51afd7ed558ccdull, x ^= x >> 29;
        return (size_t)x;
    }
};

int popcount_words(const uint64_t *w, int n) {
    int c = 0;
    for (int i = 0; i < n; ++i) c += __builtin_popcountll(w[i]);
    return c;
}

bool all_finite(const double *x, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}
}  // namespace

#define CK(call)                                                         \
    do {                                                                 \
        cudaError_t _e = (call);                                         \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call);         \
    } while (0)

namespace hb {

cudaError_t dmalloc(hb_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    DevPool &P = ctx->pool;
    bytes = (bytes + 255) / 256 * 256;
    if (bytes == 0) bytes = 256;
    if (P.base) {
        auto it = P.free_blocks.begin();
        while (it != P.free_blocks.end() && it->second < bytes) ++it;
        if (it == P.free_blocks.end()) return cudaErrorMemoryAllocation;
        const size_t off = it->first, len = it->second;
        P.free_blocks.erase(it);
        if (len > bytes) P.free_blocks[off + bytes] = len - bytes;
        *p = P.base + off;
    } else {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) return e;
    }
    P.live[*p] = bytes;
    P.live_bytes += bytes;
    P.peak_bytes = std::max(P.peak_bytes, P.live_bytes);
    return cudaSuccess;
}

void dfree(hb_ctx *ctx, void *p) {
    if (!p) return;
    DevPool &P = ctx->pool;
    auto it = P.live.find(p);
    const size_t bytes = it == P.live.end() ? 0 : it->second;
    if (it != P.live.end()) {
        P.live.erase(it);
        P.live_bytes -= bytes;
    }
    uint8_t *q = (uint8_t *)p;
    if (P.base && q >= P.base && q < P.base + P.size) {
        size_t off = (size_t)(q - P.base), len = bytes;
        auto next = P.free_blocks.lower_bound(off);
        if (next != P.free_blocks.end() && next->first == off + len) {
            len += next->second;
            next = P.free_blocks.erase(next);
        }
        if (next != P.free_blocks.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                off = prev->first;
                len += prev->second;
                P.free_blocks.erase(prev);
            }
        }
        P.free_blocks[off] = len;
    } else {
        cudaFree(p);
    }
}

}  // namespace hb

template <class T>
static int dalloc(hb_ctx *ctx, T **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = hb::dmalloc_n(ctx, p, n);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "device allocation");
    ctx->allocs.push_back(*p);
    ctx->dev_bytes += sizeof(T) * n;
    return HB_OK;
}

#define DALLOC(ptr, n)                                   \
    do {                                                 \
        int _r = dalloc(ctx, &(ptr), (size_t)(n));       \
        if (_r != HB_OK) return _r;                      \
    } while (0)

// The L2 x L2 block (classes 2 and 8) is symmetric with a full diagonal, so
// (nnz - n) / 2 entries lie below the diagonal: list each with the position
// of its mirror, so that a build evaluates only the upper triangle.  If some
// mirror were absent the lists stay unused.  One allocation, one host
// synchronisation.
static int l2_mirror_prepare(hb_ctx *ctx, int n, int W, cudaStream_t s) {
    const int64_t below = ctx->l2_nnz - n;
    if (below <= 0 || below % 2) return HB_OK;
    const int64_t nl = below / 2;
    // one allocation (each cudaMalloc costs tens of microseconds): the int64
    // lists, then every entry's column (for this search only), the lower
    // entries' columns and the flag
    uint8_t *buf = nullptr;
    const size_t n8 = (size_t)n + 1 + 2 * (size_t)nl, n4 = (size_t)ctx->l2_nnz + (size_t)nl + 1;
    int rc = dalloc(ctx, &buf, 8 * n8 + 4 * n4);
    if (rc != HB_OK) return rc;
    int64_t *low = (int64_t *)buf, *dst = low + n + 1, *src = dst + nl;
    int32_t *col_all = (int32_t *)(src + nl), *mcol = col_all + ctx->l2_nnz, *missing = mcol + nl;
    cudaError_t e = cudaMemsetAsync(missing, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(low, 0, sizeof(int64_t), s);
    l2_struct(ctx->l2, n, W, ctx->l2_rowptr, col_all, s);
    l2_lower_counts(col_all, ctx->l2_rowptr, n, low, s);
    exclusive_scan_inplace(low, n, s);
    l2_mirror_fill(col_all, ctx->l2_rowptr, n, low, nl, dst, src, mcol, missing, s);
    int32_t miss = 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&miss, missing, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "L2 mirror positions");
    if (!miss) {
        ctx->l2_low_ptr = low;
        ctx->l2_mdst = dst;
        ctx->l2_msrc = src;
        ctx->l2_mcol = mcol;
        ctx->l2_nlow = nl;
    }
    return HB_OK;
}

// l2_extra: electrons of an L2 determinant beyond the target's N (1 for the
// (N+1)-electron problem; 0 when the L2 list holds N-electron target
// determinants, as in hb_target_diag).
static int validate_problem(hb_ctx *ctx, const hb_problem *p, const hb_options *o, int l2_extra = 1) {
    if (!p) return fail(ctx, HB_ERR_INVALID_ARG, "problem is NULL");
    if (p->n_words < 1 || p->n_words > HB_MAXW)
        return fail(ctx, HB_ERR_UNSUPPORTED, "n_words must be 1..4 (up to 256 target orbitals)");
    if (p->n_to < 1 || p->n_to > 64 * p->n_words)
        return fail(ctx, HB_ERR_INVALID_ARG, "n_to must be 1..64*n_words");
    if (p->n_co < 0 || p->n_to + p->n_co >= 65535)
        return fail(ctx, HB_ERR_INVALID_ARG, "orbital count exceeds the 16-bit integral labels");
    if (p->cont_spin != HB_SPIN_ALPHA && p->cont_spin != HB_SPIN_BETA)
        return fail(ctx, HB_ERR_INVALID_ARG, "cont_spin must be HB_SPIN_ALPHA or HB_SPIN_BETA");
    if (p->n_groups < 0 || p->n_l2 < 0) return fail(ctx, HB_ERR_INVALID_ARG, "negative counts");
    if (p->n_groups > 0 && (!p->groups || p->n_co < 1))
        return fail(ctx, HB_ERR_INVALID_ARG, "groups need a continuum");
    if (p->n_elec < 1 || p->n_elec > 2 * p->n_to)
        return fail(ctx, HB_ERR_INVALID_ARG, "n_elec out of range");
    int n_energy = 0;
    for (int g = 0; g < p->n_groups && p->groups; ++g) n_energy += p->groups[g].energy != nullptr;
    if (n_energy != 0 && n_energy != p->n_groups)
        return fail(ctx, HB_ERR_INVALID_ARG, "target energies must be given for every group or for none");
    if (!p->h || !p->eri_tttt) return fail(ctx, HB_ERR_INVALID_ARG, "h or eri_tttt is NULL");
    if (p->n_groups > 0 && (!p->eri_tttc || !p->eri_ttcc || !p->eri_tctc))
        return fail(ctx, HB_ERR_INVALID_ARG, "continuum integral arrays are NULL");
    if (p->n_l2 > 0 && !p->l2_dets) return fail(ctx, HB_ERR_INVALID_ARG, "l2_dets is NULL");
    if (p->n_groups > 0 && p->n_l2 > 0 && !p->eri_tttc)
        return fail(ctx, HB_ERR_INVALID_ARG, "eri_tttc is NULL");
    if (!std::isfinite(p->e_core)) return fail(ctx, HB_ERR_INVALID_ARG, "e_core is not finite");
    if (o && o->split_tile != 0 && (o->split_tile < 3 || o->split_tile > 5))
        return fail(ctx, HB_ERR_INVALID_ARG, "split_tile must be 0, 3, 4 or 5");
    if (o && o->class4_states != 0 &&
        (o->class4_states < 4 || o->class4_states > 64 || o->class4_states % (o->class4_states > 32 ? 8 : 4)))
        return fail(ctx, HB_ERR_INVALID_ARG, "class4_states must be 0, a multiple of 4 up to 32 or of 8 up to 64");
    if (o && o->class4_threads != 0 && o->class4_threads != 32 && o->class4_threads != 64 && o->class4_threads != 128)
        return fail(ctx, HB_ERR_INVALID_ARG, "class4_threads must be 0, 32, 64 or 128");
    if (o && (o->class4_path < 0 || o->class4_path > 2))
        return fail(ctx, HB_ERR_INVALID_ARG, "class4_path must be 0, 1 or 2");
    if (o && (o->mlp_stall_iters < 0 || o->mlp_stall_iters > 1000 || o->mlp_stall_log2 < 0 || o->mlp_stall_log2 > 60))
        return fail(ctx, HB_ERR_INVALID_ARG, "mlp_stall_iters must be 0..1000 and mlp_stall_log2 0..60");
    if (o && o->diag_basis != 0 && (o->diag_basis < 3 || o->diag_basis > 10))
        return fail(ctx, HB_ERR_INVALID_ARG, "diag_basis must be 0 or 3..10");
    if (o && o->split_cols != 0 && o->split_cols != 32 && o->split_cols != 64 && o->split_cols != 128)
        return fail(ctx, HB_ERR_INVALID_ARG, "split_cols must be 0, 32, 64 or 128");
    if (o && o->split_kstage != 0 && o->split_kstage != 32 && o->split_kstage != 64)
        return fail(ctx, HB_ERR_INVALID_ARG, "split_kstage must be 0, 32 or 64");
    const int W = p->n_words, nw = 2 * W;
    // electron counts: every target determinant has the same alpha/beta split,
    // the continuum electron sets the L2 split
    int na = -1, nb = -1;
    std::unordered_set<std::vector<uint64_t>, DetHash> seen;
    const uint64_t hi_mask = p->n_to % 64 ? ((1ull << (p->n_to % 64)) - 1ull) : ~0ull;
    auto check_bits = [&](const uint64_t *d) {
        for (int s = 0; s < 2; ++s)
            for (int w = 0; w < W; ++w) {
                const int first = 64 * w;
                uint64_t allowed = first + 64 <= p->n_to ? ~0ull : (first < p->n_to ? hi_mask : 0ull);
                if (d[s * W + w] & ~allowed) return false;
            }
        return true;
    };
    for (int g = 0; g < p->n_groups; ++g) {
        const hb_group &G = p->groups[g];
        if (G.n_det < 1 || G.n_state < 1 || !G.dets || !G.ci)
            return fail(ctx, HB_ERR_INVALID_ARG, "group " + std::to_string(g) + ": empty or NULL");
        if (G.n_state > 1024)
            return fail(ctx, HB_ERR_UNSUPPORTED, "more than 1024 target states in a group");
        if (G.cont_first < 0 || G.cont_count < 1 || G.cont_first + G.cont_count > p->n_co)
            return fail(ctx, HB_ERR_INVALID_ARG, "group " + std::to_string(g) + ": continuum range");
        if (!all_finite(G.ci, (size_t)G.n_det * G.n_state))
            return fail(ctx, HB_ERR_INVALID_ARG, "group " + std::to_string(g) + ": non-finite CI");
        if (G.energy && !all_finite(G.energy, (size_t)G.n_state))
            return fail(ctx, HB_ERR_INVALID_ARG, "group " + std::to_string(g) + ": non-finite target energy");
        for (int m = 0; m < G.n_det; ++m) {
            const uint64_t *d = G.dets + (size_t)m * nw;
            if (!check_bits(d)) return fail(ctx, HB_ERR_INVALID_ARG, "determinant uses a non-target orbital");
            const int a = popcount_words(d, W), b = popcount_words(d + W, W);
            if (a + b != p->n_elec)
                return fail(ctx, HB_ERR_INVALID_ARG, "group " + std::to_string(g) + ": wrong electron count");
            if (na < 0) { na = a; nb = b; }
            if (a != na || b != nb)
                return fail(ctx, HB_ERR_INVALID_ARG, "target determinants differ in Ms (one spin coupling per problem)");
            if (!seen.insert(std::vector<uint64_t>(d, d + nw)).second)
                return fail(ctx, HB_ERR_INVALID_ARG, "duplicate target determinant (groups that share determinants "
                                                     "must have the same determinant set and continuum range and be "
                                                     "adjacent)");
        }
    }
    seen.clear();
    for (int l = 0; l < p->n_l2; ++l) {
        const uint64_t *d = p->l2_dets + (size_t)l * nw;
        if (!check_bits(d)) return fail(ctx, HB_ERR_INVALID_ARG, "L2 determinant uses a non-target orbital");
        const int a = popcount_words(d, W), b = popcount_words(d + W, W);
        if (a + b != p->n_elec + l2_extra)
            return fail(ctx, HB_ERR_INVALID_ARG, "L2 determinant with wrong electron count");
        if (na >= 0) {
            const int ea = na + (p->cont_spin == HB_SPIN_ALPHA), eb = nb + (p->cont_spin == HB_SPIN_BETA);
            if (a != ea || b != eb) return fail(ctx, HB_ERR_INVALID_ARG, "L2 determinant with a different Ms");
        }
        if (!seen.insert(std::vector<uint64_t>(d, d + nw)).second)
            return fail(ctx, HB_ERR_INVALID_ARG, "duplicate L2 determinant");
    }
    const size_t no = (size_t)(p->n_to + p->n_co);
    const size_t Pt = (size_t)p->n_to * (p->n_to + 1) / 2, ntc = (size_t)p->n_to * p->n_co;
    if (!all_finite(p->h, no * no) || !all_finite(p->eri_tttt, Pt * Pt))
        return fail(ctx, HB_ERR_INVALID_ARG, "non-finite integrals");
    for (size_t i = 0; i < no; ++i)
        for (size_t j = 0; j < i; ++j)
            if (p->h[i * no + j] != p->h[j * no + i]) return fail(ctx, HB_ERR_INVALID_ARG, "h is not symmetric");
    for (size_t i = 0; i < Pt; ++i)
        for (size_t j = 0; j < i; ++j)
            if (p->eri_tttt[i * Pt + j] != p->eri_tttt[j * Pt + i])
                return fail(ctx, HB_ERR_INVALID_ARG, "eri_tttt breaks the (pq|rs) = (rs|pq) symmetry");
    const bool deep = !o || o->validate != 0;
    if (p->n_groups > 0 || p->n_l2 > 0) {
        if (p->eri_tttc && !all_finite(p->eri_tttc, Pt * ntc)) return fail(ctx, HB_ERR_INVALID_ARG, "non-finite eri_tttc");
    }
    if (p->n_groups > 0 && deep) {
        if (!all_finite(p->eri_ttcc, Pt * (size_t)p->n_co * p->n_co) || !all_finite(p->eri_tctc, ntc * ntc))
            return fail(ctx, HB_ERR_INVALID_ARG, "non-finite continuum integrals");
        for (size_t i = 0; i < ntc; ++i)
            for (size_t j = 0; j < i; ++j)
                if (p->eri_tctc[i * ntc + j] != p->eri_tctc[j * ntc + i])
                    return fail(ctx, HB_ERR_INVALID_ARG, "eri_tctc breaks the (pq|rs) = (rs|pq) symmetry");
        const size_t nc = p->n_co;
        for (size_t k = 0; k < Pt; ++k)
            for (size_t j = 0; j < nc; ++j)
                for (size_t i = 0; i < j; ++i)
                    if (p->eri_ttcc[k * nc * nc + j * nc + i] != p->eri_ttcc[k * nc * nc + i * nc + j])
                        return fail(ctx, HB_ERR_INVALID_ARG, "eri_ttcc breaks the (pq|rs) = (pq|sr) symmetry");
    }
    return HB_OK;
}

// Validate and stage a problem; groups given over CSFs or sharing their
// determinants go through the merged-group plan (k_csf.cu) first.
static int init_context(hb_ctx *ctx, const hb_problem *p, const hb_options *o, cudaStream_t s) {
    GroupPlan plan;
    std::string err;
    int rc = prepare_groups(p, &plan, &err);
    if (rc != HB_OK) return fail(ctx, rc, err);
    if (!plan.needed) {
        rc = validate_problem(ctx, p, o);
        if (rc == HB_OK) rc = stage_problem(ctx, p, o, s);
        ctx->pool.init_allocs = ctx->allocs.size();
        return rc;
    }
    hb_problem q = *p;
    q.n_groups = (int32_t)plan.groups.size();
    q.groups = plan.groups.data();
    rc = validate_problem(ctx, &q, o);
    if (rc == HB_OK) rc = stage_problem(ctx, &q, o, s);
    if (rc != HB_OK) return rc;
    rc = expand_group_ci(ctx, plan, s, &err);
    if (rc != HB_OK) return fail(ctx, rc, err);
    ctx->user_row_off.resize(plan.user_of.size());
    for (size_t g = 0; g < plan.user_of.size(); ++g) {
        const GroupInfo &gi = ctx->groups[plan.user_of[g].first];
        ctx->user_row_off[g] = gi.row_off + (int64_t)plan.user_of[g].second * gi.cn;
    }
    ctx->pool.init_allocs = ctx->allocs.size();
    return HB_OK;
}

extern "C" int hb_init(hb_ctx **out, const hb_problem *p, const hb_options *o, void *stream) {
    if (!out) return fail(nullptr, HB_ERR_INVALID_ARG, "ctx pointer is NULL");
    *out = nullptr;
    hb_ctx *ctx = new hb_ctx();
    int rc = init_context(ctx, p, o, (cudaStream_t)stream);
    if (rc != HB_OK) { g_last_error = ctx->err; hb_destroy(ctx); return rc; }
    *out = ctx;
    return HB_OK;
}

extern "C" int hb_init_shared(hb_ctx **out, const hb_problem *p, const hb_options *o, hb_ctx *base, void *stream) {
    if (!out || !base) return fail(nullptr, HB_ERR_INVALID_ARG, "ctx pointer or base is NULL");
    *out = nullptr;
    if (base->base) return fail(nullptr, HB_ERR_INVALID_ARG, "the base context borrows its integrals itself");
    if (!p || p->n_to != base->n_to || p->n_co != base->n_co || p->n_words != base->W)
        return fail(nullptr, HB_ERR_INVALID_ARG, "problem orbitals differ from the base context");
    hb_ctx *ctx = new hb_ctx();
    ctx->base = base;
    int rc = init_context(ctx, p, o, (cudaStream_t)stream);
    if (rc != HB_OK) { g_last_error = ctx->err; hb_destroy(ctx); return rc; }
    *out = ctx;
    return HB_OK;
}

// The class of every panel label: the irrep of its target pair (r, s) for
// (jj'|rs) and of (p, q) for (jq|pj'); h and delta in class 0.
static std::vector<int32_t> label_classes(const hb_ctx *ctx, const hb_problem *p) {
    const int n_to = p->n_to, nt2 = n_to * n_to;
    const int64_t Pt = ctx->Pt;
    const int32_t *ir = p->orb_irrep;
    std::vector<int32_t> lc(ctx->K, 0);
    for (int64_t k = 0; k < Pt; ++k) {
        int r = (int)((std::sqrt(8.0 * (double)k + 1.0) - 1.0) / 2.0);
        while ((int64_t)r * (r + 1) / 2 > k) --r;
        while ((int64_t)(r + 1) * (r + 2) / 2 <= k) ++r;
        const int q = (int)(k - (int64_t)r * (r + 1) / 2);
        lc[k] = ir[r] ^ ir[q];
    }
    for (int pq = 0; pq < nt2; ++pq) lc[Pt + pq] = ir[pq / n_to] ^ ir[pq % n_to];
    return lc;
}

// Panel label classes: one class of every label without orbital symmetry;
// with it, the labels of each irrep of the target pair in ascending order,
// Kc (the largest class, padded to 64) columns per class.  A context that
// borrows its integrals borrows these.
static int setup_label_classes(hb_ctx *ctx, const hb_problem *p, cudaStream_t s) {
    const int delta_label = (int)(ctx->Pt + (int64_t)p->n_to * p->n_to + 1);
    if (ctx->base) {
        const hb_ctx *B = ctx->base;
        if ((p->orb_irrep != nullptr) != (B->n_cls > 1))
            return fail(ctx, HB_ERR_INVALID_ARG, "orb_irrep must be given for the base context and this one alike");
        ctx->n_cls = B->n_cls; ctx->Kc = B->Kc; ctx->cls_labels = B->cls_labels; ctx->cls_labels_h = B->cls_labels_h;
        ctx->co_irrep = B->co_irrep; ctx->co_irrep_d = B->co_irrep_d; ctx->delta_pos = B->delta_pos;
    } else if (!p->orb_irrep) {
        ctx->n_cls = 1;
        ctx->Kc = ctx->Kpad;
        ctx->delta_pos = delta_label;
    } else {
        const int n_orb = p->n_to + p->n_co;
        for (int i = 0; i < n_orb; ++i)
            if (p->orb_irrep[i] < 0 || p->orb_irrep[i] > 7)
                return fail(ctx, HB_ERR_INVALID_ARG, "orb_irrep values must be 0..7");
        const std::vector<int32_t> lc = label_classes(ctx, p);
        std::vector<std::vector<int32_t>> lists(8);
        for (int k = 0; k < ctx->K; ++k) lists[lc[k]].push_back(k);
        size_t most = 1;
        for (auto &l : lists) most = std::max(most, l.size());
        ctx->n_cls = 8;
        ctx->Kc = (int)((most + 63) / 64 * 64);
        ctx->cls_labels_h.assign((size_t)8 * ctx->Kc, -1);
        for (int x = 0; x < 8; ++x)
            for (size_t i = 0; i < lists[x].size(); ++i) {
                ctx->cls_labels_h[(size_t)x * ctx->Kc + i] = lists[x][i];
                if (lists[x][i] == delta_label) ctx->delta_pos = (int)i;
            }
        ctx->co_irrep.assign(p->orb_irrep + p->n_to, p->orb_irrep + n_orb);
        DALLOC(ctx->cls_labels, (size_t)8 * ctx->Kc);
        DALLOC(ctx->co_irrep_d, std::max(p->n_co, 1));
        CK(cudaMemcpyAsync(ctx->cls_labels, ctx->cls_labels_h.data(), sizeof(int32_t) * ctx->cls_labels_h.size(),
                           cudaMemcpyHostToDevice, s));
        if (p->n_co > 0)
            CK(cudaMemcpyAsync(ctx->co_irrep_d, ctx->co_irrep.data(), sizeof(int32_t) * p->n_co,
                               cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));   // the host tables are staged from (pageable) vectors
    }
    if (ctx->n_cls > 1)
        for (int g = 0; g < p->n_groups; ++g) {
            const hb_group &G = p->groups[g];
            if (G.cont_count < 0 || G.cont_first < 0 || (int64_t)G.cont_first + G.cont_count > p->n_co)
                return fail(ctx, HB_ERR_INVALID_ARG, "group " + std::to_string(g) + ": continuum range");
            for (int j = G.cont_first; j < G.cont_first + G.cont_count; ++j)
                if (ctx->co_irrep[j] != ctx->co_irrep[G.cont_first])
                    return fail(ctx, HB_ERR_INVALID_ARG,
                                "group " + std::to_string(g) + ": its continuum range spans several irreps");
        }
    return HB_OK;
}

int stage_problem(hb_ctx *ctx, const hb_problem *p, const hb_options *o, cudaStream_t s) {
    CK(cudaGetDevice(&ctx->device));
    ctx->n_to = p->n_to; ctx->n_co = p->n_co; ctx->n_orb = p->n_to + p->n_co;
    ctx->n_elec = p->n_elec; ctx->W = p->n_words; ctx->cont_spin = p->cont_spin;
    ctx->n_groups = p->n_groups; ctx->n_l2 = p->n_l2; ctx->e_core = p->e_core;
    ctx->split_slices = (o && o->split_slices > 0) ? o->split_slices : 6;
    ctx->autotune = (o && o->autotune) ? 1 : 0;
    if (o) {
        ctx->force_tile = o->split_tile;
        ctx->force_cols = o->split_cols;
        ctx->force_kstage = o->split_kstage;
        ctx->force_c4_states = o->class4_states;
        ctx->force_c4_threads = o->class4_threads;
        ctx->c4_path = o->class4_path;
        if (o->mlp_stall_iters > 0) ctx->stall_iters = o->mlp_stall_iters;
        if (o->mlp_stall_log2 > 0) ctx->stall_log2 = o->mlp_stall_log2;
        if (o->diag_basis > 0) ctx->diag_basis = o->diag_basis;
    }
    ctx->Pt = (int64_t)p->n_to * (p->n_to + 1) / 2;
    ctx->K = (int)(ctx->Pt + (int64_t)p->n_to * p->n_to + 2);
    ctx->Kpad = (ctx->K + 63) / 64 * 64;
    const int W = ctx->W, nw = 2 * W;
    const bool validate = !o || o->validate;
    // the expansion panel's label classes (orbital symmetry)
    {
        int rc = setup_label_classes(ctx, p, s);
        if (rc != HB_OK) return rc;
    }
    // groups and offsets
    int64_t det_off = 0, ci_off = 0, row_off = 0, e_off = 0;
    for (int g = 0; g < p->n_groups; ++g) {
        const hb_group &G = p->groups[g];
        GroupInfo gi;
        gi.ndet = G.n_det; gi.ns = G.n_state; gi.cf = G.cont_first; gi.cn = G.cont_count;
        gi.det_off = det_off; gi.ci_off = ci_off; gi.row_off = row_off; gi.e_off = e_off;
        ctx->groups.push_back(gi);
        det_off += (int64_t)G.n_det * nw;
        ci_off += (int64_t)G.n_det * G.n_state;
        row_off += (int64_t)G.n_state * G.cont_count;
        e_off += G.n_state;
    }
    ctx->Dc = row_off;
    ctx->dim = row_off + p->n_l2;
    const size_t no = ctx->n_orb, Pt = ctx->Pt, ntc = (size_t)p->n_to * p->n_co, ncc = (size_t)p->n_co * p->n_co;
    // --- stage integrals, determinants, CI
    const bool shared = ctx->base != nullptr;
    if (shared) {
        // integrals, their tables and the expansion panel belong to the base context
        ctx->h = ctx->base->h; ctx->tttt = ctx->base->tttt; ctx->tttc = ctx->base->tttc;
        ctx->jk = ctx->base->jk; ctx->panel = ctx->base->panel;
    } else {
        DALLOC(ctx->h, no * no);
        DALLOC(ctx->tttt, Pt * Pt);
        DALLOC(ctx->jk, 2 * (size_t)p->n_to * p->n_to);
        CK(cudaMemcpyAsync(ctx->h, p->h, sizeof(double) * no * no, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->tttt, p->eri_tttt, sizeof(double) * Pt * Pt, cudaMemcpyHostToDevice, s));
        if (p->eri_tttc && ntc > 0) {
            DALLOC(ctx->tttc, Pt * ntc);
            CK(cudaMemcpyAsync(ctx->tttc, p->eri_tttc, sizeof(double) * Pt * ntc, cudaMemcpyHostToDevice, s));
        }
    }
    DALLOC(ctx->dets, std::max<int64_t>(det_off, 1));
    DALLOC(ctx->ci, std::max<int64_t>(ci_off, 1));
    for (int g = 0; g < p->n_groups; ++g) {
        const hb_group &G = p->groups[g];
        const GroupInfo &gi = ctx->groups[g];
        CK(cudaMemcpyAsync(ctx->dets + gi.det_off, G.dets, sizeof(uint64_t) * G.n_det * nw, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->ci + gi.ci_off, G.ci, sizeof(double) * G.n_det * G.n_state, cudaMemcpyHostToDevice, s));
    }
    if (p->n_groups > 0 && p->groups[0].energy) {
        DALLOC(ctx->energy, e_off);
        for (int g = 0; g < p->n_groups; ++g)
            CK(cudaMemcpyAsync(ctx->energy + ctx->groups[g].e_off, p->groups[g].energy,
                               sizeof(double) * p->groups[g].n_state, cudaMemcpyHostToDevice, s));
    }
    DALLOC(ctx->l2, std::max(p->n_l2, 1) * nw);
    if (p->n_l2 > 0)
        CK(cudaMemcpyAsync(ctx->l2, p->l2_dets, sizeof(uint64_t) * p->n_l2 * nw, cudaMemcpyHostToDevice, s));
    Ints I = ctx->ints();
    if (!shared) build_jk(I, ctx->jk, s);
    // --- the expansion panel (classes 1,3,5,6,7)
    if (p->n_groups > 0 && !shared) {
        DALLOC(ctx->panel, ncc * ctx->Kc);
        double *t_ttcc = nullptr, *t_tctc = nullptr;
        CK(cudaMalloc(&t_ttcc, sizeof(double) * Pt * ncc));
        cudaError_t e2 = cudaMalloc(&t_tctc, sizeof(double) * ntc * ntc);
        if (e2 != cudaSuccess) { cudaFree(t_ttcc); return cuda_fail(ctx, e2, "cudaMalloc"); }
        cudaError_t e3 = cudaMemcpyAsync(t_ttcc, p->eri_ttcc, sizeof(double) * Pt * ncc, cudaMemcpyHostToDevice, s);
        if (e3 == cudaSuccess)
            e3 = cudaMemcpyAsync(t_tctc, p->eri_tctc, sizeof(double) * ntc * ntc, cudaMemcpyHostToDevice, s);
        int sym_bad = 0;
        if (e3 == cudaSuccess) {
            build_panel(t_ttcc, t_tctc, ctx->h, p->n_to, p->n_co, ctx->Kc, ctx->n_cls > 1 ? ctx->cls_labels : nullptr,
                        ctx->co_irrep_d, ctx->panel, s);
            if (ctx->n_cls > 1 && validate) {
                // every panel value outside its row's class must vanish
                int32_t *lcls = nullptr;
                int *flag = nullptr;
                e3 = cudaMalloc(&lcls, sizeof(int32_t) * ctx->K);
                if (e3 == cudaSuccess) e3 = cudaMalloc(&flag, sizeof(int));
                std::vector<int32_t> lc = label_classes(ctx, p);
                if (e3 == cudaSuccess)
                    e3 = cudaMemcpyAsync(lcls, lc.data(), sizeof(int32_t) * ctx->K, cudaMemcpyHostToDevice, s);
                if (e3 == cudaSuccess) e3 = cudaMemsetAsync(flag, 0, sizeof(int), s);
                if (e3 == cudaSuccess) {
                    check_panel_symmetry(t_ttcc, t_tctc, ctx->h, p->n_to, p->n_co, ctx->K, lcls, ctx->co_irrep_d,
                                         flag, s);
                    e3 = cudaMemcpyAsync(&sym_bad, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
                }
                if (e3 == cudaSuccess) e3 = cudaStreamSynchronize(s);
                cudaFree(lcls);
                cudaFree(flag);
            }
            if (e3 == cudaSuccess) e3 = cudaStreamSynchronize(s);
        }
        cudaFree(t_ttcc);
        cudaFree(t_tctc);
        if (e3 != cudaSuccess) return cuda_fail(ctx, e3, "panel staging");
        if (sym_bad)
            return fail(ctx, HB_ERR_INVALID_ARG,
                        "orb_irrep: an integral of the continuum classes breaks the declared symmetry");
    }
    // --- classification counts (structure of every class)
    for (int g = 0; g < p->n_groups; ++g)
        for (int gp = 0; gp <= g; ++gp) {
            GroupPair P;
            P.g = g; P.gp = gp; P.same = (g == gp);
            DALLOC(P.rowptr, ctx->groups[g].ndet + 1);
            ctx->gps.push_back(P);
        }
    for (auto &P : ctx->gps) {
        const GroupInfo &A = ctx->groups[P.g], &B = ctx->groups[P.gp];
        CK(cudaMemsetAsync(P.rowptr, 0, sizeof(int64_t), s));
        k1_count(ctx->dets + A.det_off, A.ndet, ctx->dets + B.det_off, B.ndet, W, 0, 2, 0, P.rowptr, s);
        exclusive_scan_inplace(P.rowptr, A.ndet, s);
        DALLOC(P.seg_off, (int64_t)A.ndet * seg_count(B.ndet));
        k1_seg_offsets(ctx->dets + A.det_off, A.ndet, ctx->dets + B.det_off, B.ndet, W, 0, 2, 0, P.seg_off, s);
    }
    for (int g = 0; g < p->n_groups; ++g) {
        GroupL2 L;
        DALLOC(L.rowptr, p->n_l2 + 1);
        CK(cudaMemsetAsync(L.rowptr, 0, sizeof(int64_t), s));
        k1_count(ctx->l2, p->n_l2, ctx->dets + ctx->groups[g].det_off, ctx->groups[g].ndet, W, 1, 2, 0, L.rowptr, s);
        exclusive_scan_inplace(L.rowptr, p->n_l2, s);
        DALLOC(L.seg_off, (int64_t)std::max(p->n_l2, 1) * seg_count(ctx->groups[g].ndet));
        k1_seg_offsets(ctx->l2, p->n_l2, ctx->dets + ctx->groups[g].det_off, ctx->groups[g].ndet, W, 1, 2, 0,
                       L.seg_off, s);
        ctx->gl2.push_back(L);
    }
    DALLOC(ctx->l2_rowptr, p->n_l2 + 1);
    CK(cudaMemsetAsync(ctx->l2_rowptr, 0, sizeof(int64_t), s));
    k1_count(ctx->l2, p->n_l2, ctx->l2, p->n_l2, W, 0, 2, 0, ctx->l2_rowptr, s);
    exclusive_scan_inplace(ctx->l2_rowptr, p->n_l2, s);
    DALLOC(ctx->l2_seg_off, (int64_t)std::max(p->n_l2, 1) * seg_count(p->n_l2));
    k1_seg_offsets(ctx->l2, p->n_l2, ctx->l2, p->n_l2, W, 0, 2, 0, ctx->l2_seg_off, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    ctx->tt_pairs = 0;
    for (auto &P : ctx->gps) {
        CK(cudaMemcpy(&P.n_pairs, P.rowptr + ctx->groups[P.g].ndet, sizeof(int64_t), cudaMemcpyDeviceToHost));
        ctx->tt_pairs += P.n_pairs;
    }
    ctx->tl2_pairs = 0;
    for (auto &L : ctx->gl2) {
        CK(cudaMemcpy(&L.n_pairs, L.rowptr + p->n_l2, sizeof(int64_t), cudaMemcpyDeviceToHost));
        ctx->tl2_pairs += L.n_pairs;
    }
    CK(cudaMemcpy(&ctx->l2_nnz, ctx->l2_rowptr + p->n_l2, sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (p->n_l2 > 1 && ctx->l2_nnz > 0) {
        const int rc = l2_mirror_prepare(ctx, p->n_l2, W, s);
        if (rc != HB_OK) return rc;
    }
    // --- per group pair scratch; the gamma item count needs the records
    const int n_keys = 2 * p->n_to * p->n_to;
    for (auto &P : ctx->gps) {
        const GroupInfo &A = ctx->groups[P.g], &B = ctx->groups[P.gp];
        DALLOC(P.pairs, P.n_pairs);
        DALLOC(P.val, P.n_pairs);
        DALLOC(P.item_ptr, A.ndet + 1);
        k1_fill_pairs(ctx->dets + A.det_off, A.ndet, ctx->dets + B.det_off, B.ndet, W, 0, ctx->cont_spin, 2, 0,
                      P.rowptr, P.pairs, s);
        CK(cudaMemsetAsync(P.item_ptr, 0, sizeof(int64_t), s));
        gamma_item_counts(P.pairs, P.rowptr, A.ndet, ctx->n_elec, P.item_ptr, s);
        exclusive_scan_inplace(P.item_ptr, A.ndet, s);
        CK(cudaMemcpyAsync(&P.n_items, P.item_ptr + A.ndet, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        P.n_chunks = sort_chunks(P.n_items, n_keys);
        DALLOC(P.items, P.n_items);
        DALLOC(P.order, P.n_items);
        DALLOC(P.sort_off, (int64_t)n_keys * P.n_chunks + 1);
        DALLOC(P.sort_cur, (int64_t)n_keys * P.n_chunks + 1);
        DALLOC(P.sort_part, blocks_scan((int64_t)n_keys * P.n_chunks) + 1);
        const int64_t nout = (int64_t)A.ns * B.ns;
        DALLOC(P.gamma, n_keys * nout);
        DALLOC(P.W, (int64_t)A.ndet * B.ns);
        DALLOC(P.partial, (int64_t)tn_chunks(A.ndet) * nout);
        DALLOC(P.partial_s, P.same ? (int64_t)tn_chunks(A.ndet) * nout : 1);
        DALLOC(P.gdiag, P.same ? (int64_t)tn_chunks(A.ndet) * 2 * p->n_to * nout : 1);
        DALLOC(P.S, nout);
        DALLOC(P.E, nout);
        std::vector<int32_t> nn;
        for (int a = 0; a < A.ns; ++a)
            for (int b = 0; b < B.ns; ++b)
                if (!P.same || b <= a) { nn.push_back(a); nn.push_back(b); }
        P.n_nn = (int)(nn.size() / 2);
        DALLOC(P.nn, nn.size());
        CK(cudaMemcpyAsync(P.nn, nn.data(), sizeof(int32_t) * nn.size(), cudaMemcpyHostToDevice, s));
        DALLOC(P.A, (int64_t)P.n_nn * ctx->Kpad);
        CK(cudaStreamSynchronize(s));
    }
    for (auto &L : ctx->gl2) DALLOC(L.pairs, L.n_pairs);
    CK(cudaStreamSynchronize(s));
    return HB_OK;
}

int ensure_df(hb_ctx *ctx, cudaStream_t s) {
    if (ctx->ci_df) return HB_OK;
    const size_t no = ctx->n_orb, ntc = (size_t)ctx->n_to * ctx->n_co;
    if (ctx->base) {
        int rc = ensure_df(ctx->base, s);
        if (rc != HB_OK) return fail(ctx, rc, ctx->base->err);
        ctx->tttc_df = ctx->base->tttc_df;
        ctx->h_df = ctx->base->h_df;
        ctx->tttt_df = ctx->base->tttt_df;
        ctx->jk_df = ctx->base->jk_df;
    } else {
        DALLOC(ctx->h_df, no * no);
        split_df(ctx->h, (int64_t)(no * no), ctx->h_df, s);
        DALLOC(ctx->tttt_df, (size_t)ctx->Pt * ctx->Pt);
        split_df(ctx->tttt, ctx->Pt * ctx->Pt, ctx->tttt_df, s);
        DALLOC(ctx->jk_df, 2 * (size_t)ctx->n_to * ctx->n_to);
        split_df(ctx->jk, 2 * (int64_t)ctx->n_to * ctx->n_to, ctx->jk_df, s);
        if (ctx->tttc && ntc > 0) {
            DALLOC(ctx->tttc_df, (size_t)ctx->Pt * ntc);
            split_df(ctx->tttc, (int64_t)((size_t)ctx->Pt * ntc), ctx->tttc_df, s);
        }
    }
    for (auto &P : ctx->gps) DALLOC(P.A_df, (int64_t)P.n_nn * ctx->Kpad);
    int64_t nci = 0;
    for (auto &g : ctx->groups) nci += (int64_t)g.ndet * g.ns;
    DALLOC(ctx->ci_df, std::max<int64_t>(nci, 1));
    split_df(ctx->ci, nci, ctx->ci_df, s);
    CK(cudaGetLastError());
    return HB_OK;
}

extern "C" int hb_query(const hb_ctx *ctx, hb_layout *out) {
    if (!ctx || !out) return fail(nullptr, HB_ERR_INVALID_ARG, "NULL argument");
    out->dim = ctx->dim;
    out->contracted_dim = ctx->Dc;
    out->n_l2 = ctx->n_l2;
    out->l2_nnz = ctx->l2_nnz;
    out->tt_pairs = ctx->tt_pairs;
    out->tl2_pairs = ctx->tl2_pairs;
    out->n_labels = ctx->K;
    out->device_bytes = (int64_t)ctx->dev_bytes;
    out->workspace_bytes = ctx->pool.measured;
    out->n_groups = ctx->n_groups;
    out->n_words = ctx->W;
    return HB_OK;
}

extern "C" int64_t hb_group_offset(const hb_ctx *ctx, int32_t g) {
    if (!ctx || g < 0) return -1;
    if (!ctx->user_row_off.empty()) {
        const int32_t n = (int32_t)ctx->user_row_off.size();
        if (g > n) return -1;
        return g == n ? ctx->Dc : ctx->user_row_off[g];
    }
    if (g > ctx->n_groups) return -1;
    return g == ctx->n_groups ? ctx->Dc : ctx->groups[g].row_off;
}

extern "C" int hb_build_blocks(hb_ctx *ctx, int32_t precision, const hb_blocks *out, hb_stats *st,
                               void *stream) {
    if (!ctx || !out) return fail(ctx, HB_ERR_INVALID_ARG, "NULL argument");
    if (precision != HB_FP64 && precision != HB_MIXED)
        return fail(ctx, HB_ERR_INVALID_ARG, "precision must be HB_FP64 or HB_MIXED");
    if (ctx->Dc > 0 && !out->Hcc) return fail(ctx, HB_ERR_INVALID_ARG, "Hcc is NULL");
    if (ctx->Dc > 0 && ctx->n_l2 > 0 && !out->Hlc) return fail(ctx, HB_ERR_INVALID_ARG, "Hlc is NULL");
    if (ctx->n_l2 > 0 && (!out->l2_row_ptr || !out->l2_col || !out->l2_val))
        return fail(ctx, HB_ERR_INVALID_ARG, "L2 CSR arrays are NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    // the build as a plan of grouped launches over this context's group pairs,
    // kept between builds (made again for another precision, re-pointed for
    // other output blocks)
    hb::Plan *plan = (hb::Plan *)ctx->plan;
    std::string err;
    if (plan && plan_precision(plan) != precision) {
        cudaStreamSynchronize(s);
        plan_destroy(plan);
        plan = nullptr;
        ctx->plan = nullptr;
    }
    if (!plan) {
        hb_ctx *one[1] = {ctx};
        int rc = plan_create(one, 1, out, precision, &plan, &err, s);
        if (rc != HB_OK) return fail(ctx, rc, err);
        ctx->plan = plan;
        if (ctx->autotune) {
            rc = plan_autotune(plan, s, &err);
            if (rc != HB_OK) return fail(ctx, rc, err);
        }
    } else if (!plan_outputs_equal(plan, out)) {
        int rc = plan_set_outputs(plan, out, &err, s);
        if (rc != HB_OK) return fail(ctx, rc, err);
    }
    int launches = 0;
    int rc = plan_run(plan, s, true, false, &launches, &err);
    if (rc != HB_OK) return fail(ctx, rc, err);
    if (precision == HB_MIXED) {
        // the tensor-core kernel reports a bounded-wait timeout in a device word
        int word = 0;
        CK(cudaStreamSynchronize(s));
        if (plan_error_word(plan, &word) != HB_OK) return fail(ctx, HB_ERR_CUDA, "reading the mixed error word");
        if (word != 0)
            return fail(ctx, HB_ERR_TIMEOUT, "a tensor-core kernel (split expansion, codes 1-6, or class 4, codes 21-26) gave up waiting (code " + std::to_string(word) + ")");
    }
    if (st) plan_stats(plan, st);
    return HB_OK;
}

extern "C" int hb_target_diag(const hb_problem *p, int32_t g, int32_t k, double tol, int32_t max_iter,
                              double *energies, double *ci, hb_stats *st, void *stream) {
    if (!p || !energies || !ci) return fail(nullptr, HB_ERR_INVALID_ARG, "NULL argument");
    if (g < 0 || g >= p->n_groups || !p->groups) return fail(nullptr, HB_ERR_INVALID_ARG, "group out of range");
    const hb_group &G = p->groups[g];
    if (k < 1 || k > G.n_det || !G.dets) return fail(nullptr, HB_ERR_INVALID_ARG, "k must be 1..n_det");
    // The target Hamiltonian over the group's determinants is the L2-L2 block
    // (classes 2 and 8) of a problem whose L2 list is those N-electron
    // determinants and which has no target group.
    hb_problem q{};
    q.n_to = p->n_to; q.n_co = p->n_co; q.n_elec = p->n_elec; q.n_words = p->n_words; q.cont_spin = p->cont_spin;
    q.h = p->h; q.eri_tttt = p->eri_tttt;
    q.n_groups = 0; q.groups = nullptr;
    q.n_l2 = G.n_det; q.l2_dets = G.dets; q.e_core = p->e_core;
    hb_options o{};
    o.validate = 1;
    hb_ctx *ctx = new hb_ctx();
    int rc = validate_problem(ctx, &q, &o, 0);
    if (rc == HB_OK) rc = stage_problem(ctx, &q, &o, (cudaStream_t)stream);
    if (rc != HB_OK) { g_last_error = ctx->err; hb_destroy(ctx); return rc; }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = G.n_det, nnz = std::max<int64_t>(ctx->l2_nnz, 1);
    hb_blocks H{};
    double *evecs = nullptr;
    cudaError_t e = cudaMalloc((void **)&H.l2_row_ptr, sizeof(int64_t) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&H.l2_col, sizeof(int32_t) * nnz);
    if (e == cudaSuccess) e = cudaMalloc((void **)&H.l2_val, sizeof(double) * nnz);
    if (e == cudaSuccess) e = cudaMalloc((void **)&evecs, sizeof(double) * n * k);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaMalloc");
    if (rc == HB_OK) rc = hb_build_blocks(ctx, HB_FP64, &H, nullptr, stream);
    int rc_diag = HB_OK;
    std::vector<double> V;
    if (rc == HB_OK) {
        rc_diag = hb_diag(ctx, &H, k, tol, max_iter, HB_PRECOND_DIAG, nullptr, energies, evecs, st, stream);
        if (rc_diag == HB_OK || rc_diag == HB_ERR_NOT_CONVERGED) {
            V.resize((size_t)n * k);
            e = cudaMemcpyAsync(V.data(), evecs, sizeof(double) * n * k, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "eigenvector readback");
        } else {
            rc = rc_diag;
        }
    }
    if (rc == HB_OK) {
        // a fixed sign per column: its largest-magnitude entry positive
        for (int c = 0; c < k; ++c) {
            int64_t best = 0;
            for (int64_t i = 1; i < n; ++i)
                if (std::fabs(V[i * k + c]) > std::fabs(V[best * k + c])) best = i;
            const double sg = V[best * k + c] < 0 ? -1.0 : 1.0;
            for (int64_t i = 0; i < n; ++i) ci[i * k + c] = sg * V[i * k + c];
        }
        rc = rc_diag;
    }
    if (rc != HB_OK) g_last_error = ctx->err;
    cudaFree(H.l2_row_ptr);
    cudaFree(H.l2_col);
    cudaFree(H.l2_val);
    cudaFree(evecs);
    hb_destroy(ctx);
    return rc;
}

// ------------------------------------------------------------ sharded build

extern "C" int hb_shard_coef_len(const hb_ctx *ctx, int64_t *len) {
    if (!ctx || !len) return fail(nullptr, HB_ERR_INVALID_ARG, "NULL argument");
    int64_t n = 0;
    for (auto &P : ctx->gps) n += (int64_t)P.n_nn * ctx->Kpad;
    *len = n;
    return HB_OK;
}

// The cached plan of this context's share (rank of nranks), pointed at out.
static int shard_plan(hb_ctx *ctx, int precision, int rank, int nranks, const hb_blocks *out, hb::Plan **plan,
                      cudaStream_t s) {
    std::string err;
    hb::Plan *p = (hb::Plan *)ctx->shard_plan;
    if (p && !plan_is_shard(p, precision, rank, nranks)) {
        cudaStreamSynchronize(s);
        plan_destroy(p);
        p = nullptr;
        ctx->shard_plan = nullptr;
    }
    if (!p) {
        hb_ctx *one[1] = {ctx};
        int rc = plan_create(one, 1, out, precision, &p, &err, s, rank, nranks);
        if (rc != HB_OK) return fail(ctx, rc, err);
        ctx->shard_plan = p;
    } else if (!plan_outputs_equal(p, out)) {
        int rc = plan_set_outputs(p, out, &err, s);
        if (rc != HB_OK) return fail(ctx, rc, err);
    }
    *plan = p;
    return HB_OK;
}

static int shard_args(hb_ctx *ctx, int precision, int rank, int nranks) {
    if (precision != HB_FP64 && precision != HB_MIXED)
        return fail(ctx, HB_ERR_INVALID_ARG, "precision must be HB_FP64 or HB_MIXED");
    if (nranks < 1 || rank < 0 || rank >= nranks) return fail(ctx, HB_ERR_INVALID_ARG, "need 0 <= rank < nranks");
    return HB_OK;
}

extern "C" int hb_build_contract(hb_ctx *ctx, int32_t precision, int32_t rank, int32_t nranks, double *partial,
                                 hb_stats *st, void *stream) {
    if (!ctx) return fail(nullptr, HB_ERR_INVALID_ARG, "NULL argument");
    int rc = shard_args(ctx, precision, rank, nranks);
    if (rc != HB_OK) return rc;
    int64_t len = 0;
    hb_shard_coef_len(ctx, &len);
    if (len > 0 && !partial) return fail(ctx, HB_ERR_INVALID_ARG, "partial is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    // the contraction writes no output block: a cached plan of this share is
    // used as it is, a new one is made without outputs
    hb::Plan *p = (hb::Plan *)ctx->shard_plan;
    if (!p || !plan_is_shard(p, precision, rank, nranks)) {
        hb_blocks none{};
        rc = shard_plan(ctx, precision, rank, nranks, &none, &p, s);
        if (rc != HB_OK) return rc;
    }
    // the stage timers belong to whole builds: this phase runs untimed
    plan_set_phase(p, 1);
    std::string err;
    int launches = 0;
    rc = plan_run(p, s, false, false, &launches, &err);
    plan_set_phase(p, 0);
    if (rc != HB_OK) return fail(ctx, rc, err);
    // this rank's contracted coefficient rows, group pair after group pair
    int64_t off = 0;
    for (auto &P : ctx->gps) {
        const size_t n = (size_t)P.n_nn * ctx->Kpad;
        CK(cudaMemcpyAsync(partial + off, P.A, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        off += (int64_t)n;
    }
    if (st) {
        memset(st, 0, sizeof(*st));
        st->kernel_launches = launches;
    }
    return HB_OK;
}

extern "C" int hb_build_expand(hb_ctx *ctx, int32_t precision, int32_t rank, int32_t nranks, const double *reduced,
                               const hb_blocks *out, hb_stats *st, void *stream) {
    if (!ctx || !out) return fail(ctx, HB_ERR_INVALID_ARG, "NULL argument");
    int rc = shard_args(ctx, precision, rank, nranks);
    if (rc != HB_OK) return rc;
    int64_t len = 0;
    hb_shard_coef_len(ctx, &len);
    if (len > 0 && !reduced) return fail(ctx, HB_ERR_INVALID_ARG, "reduced is NULL");
    if (ctx->Dc > 0 && !out->Hcc) return fail(ctx, HB_ERR_INVALID_ARG, "Hcc is NULL");
    if (ctx->Dc > 0 && ctx->n_l2 > 0 && !out->Hlc) return fail(ctx, HB_ERR_INVALID_ARG, "Hlc is NULL");
    if (ctx->n_l2 > 0 && (!out->l2_row_ptr || !out->l2_col || !out->l2_val))
        return fail(ctx, HB_ERR_INVALID_ARG, "L2 CSR arrays are NULL");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    hb::Plan *p = nullptr;
    rc = shard_plan(ctx, precision, rank, nranks, out, &p, s);
    if (rc != HB_OK) return rc;
    // the summed coefficient rows of all ranks in place of this rank's
    int64_t off = 0;
    for (auto &P : ctx->gps) {
        const size_t n = (size_t)P.n_nn * ctx->Kpad;
        CK(cudaMemcpyAsync(P.A, reduced + off, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        if (precision == HB_MIXED && P.A_df) split_df(P.A, (int64_t)n, P.A_df, s);
        off += (int64_t)n;
    }
    plan_set_phase(p, 2);
    std::string err;
    int launches = 0;
    rc = plan_run(p, s, false, false, &launches, &err);
    plan_set_phase(p, 0);
    if (rc != HB_OK) return fail(ctx, rc, err);
    if (precision == HB_MIXED) {
        int word = 0;
        CK(cudaStreamSynchronize(s));
        if (plan_error_word(p, &word) != HB_OK) return fail(ctx, HB_ERR_CUDA, "reading the mixed error word");
        if (word != 0) return fail(ctx, HB_ERR_TIMEOUT, "a tensor-core kernel gave up waiting (code " + std::to_string(word) + ")");
    }
    if (st) {
        memset(st, 0, sizeof(*st));
        st->kernel_launches = launches;
    }
    return HB_OK;
}

extern "C" int hb_workspace_size(hb_ctx *ctx, int32_t precision, int32_t diag_k, int32_t precond, int64_t *bytes,
                                 void *stream) {
    if (!ctx || !bytes) return fail(ctx, HB_ERR_INVALID_ARG, "NULL argument");
    if (precision != HB_FP64 && precision != HB_MIXED && precision != -1)
        return fail(ctx, HB_ERR_INVALID_ARG, "precision must be HB_FP64, HB_MIXED or -1 (no build)");
    if (diag_k < 0) return fail(ctx, HB_ERR_INVALID_ARG, "diag_k < 0");
    if (ctx->pool.base) return fail(ctx, HB_ERR_INVALID_ARG, "a workspace is already set");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    // measure from nothing: the build's own set-up (plan, double-float copies,
    // tensor-core slices and tables) runs under the byte count, then goes again
    release_lazy(ctx);
    const size_t live0 = ctx->pool.live_bytes;
    ctx->pool.peak_bytes = live0;
    if (precision != -1) {
        hb_blocks none{};
        hb_ctx *one[1] = {ctx};
        hb::Plan *plan = nullptr;
        std::string err;
        int rc = plan_create(one, 1, &none, precision, &plan, &err, s);
        if (rc != HB_OK) { release_lazy(ctx); return fail(ctx, rc, err); }
        cudaStreamSynchronize(s);
        plan_destroy(plan);
    }
    // the build's set-up stays while a solve runs, so the two add up
    int64_t need = (int64_t)(ctx->pool.peak_bytes - live0);
    release_lazy(ctx);
    if (diag_k > 0) need += diag_workspace_bytes(ctx, diag_k, precond);
    // the autotuner's timing buffers and the allocator's alignment
    need += (16 << 20) + need / 64;
    ctx->pool.measured = need;
    *bytes = need;
    return HB_OK;
}

extern "C" int hb_set_workspace(hb_ctx *ctx, void *dev_ptr, size_t bytes) {
    if (!ctx || !dev_ptr || bytes < 256) return fail(ctx, HB_ERR_INVALID_ARG, "NULL or empty workspace");
    if (ctx->pool.base) return fail(ctx, HB_ERR_INVALID_ARG, "a workspace is already set");
    CK(cudaSetDevice(ctx->device));
    // what a previous build or solve set up with cudaMalloc goes; it is made
    // again inside the workspace on next use
    release_lazy(ctx);
    const uintptr_t a = (uintptr_t)dev_ptr, a256 = (a + 255) / 256 * 256;
    if (a256 - a >= bytes) return fail(ctx, HB_ERR_INVALID_ARG, "workspace too small");
    ctx->pool.base = (uint8_t *)a256;
    ctx->pool.size = (bytes - (a256 - a)) / 256 * 256;
    ctx->pool.free_blocks.clear();
    ctx->pool.free_blocks[0] = ctx->pool.size;
    return HB_OK;
}

extern "C" int hb_classify(const uint64_t *a, int32_t n_a, const uint64_t *b, int32_t n_b, int32_t n_words,
                           int32_t mode, int32_t cont_spin, int32_t max_degree, int32_t lower, int64_t *row_ptr,
                           hb_pair *pairs, int64_t cap, int64_t *total, void *stream) {
    hb_ctx *ctx = nullptr;
    if (n_words < 1 || n_words > HB_MAXW) return fail(ctx, HB_ERR_UNSUPPORTED, "n_words must be 1..4");
    if (n_a < 0 || n_b < 0 || !row_ptr || !total || (mode != 0 && mode != 1) || max_degree < 0)
        return fail(ctx, HB_ERR_INVALID_ARG, "bad classify arguments");
    if ((n_a > 0 && !a) || (n_b > 0 && !b)) return fail(ctx, HB_ERR_INVALID_ARG, "NULL determinant list");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s));
    if (n_a > 0) {
        k1_count(a, n_a, b, n_b, n_words, mode, max_degree, lower, row_ptr, s);
        exclusive_scan_inplace(row_ptr, n_a, s);
    }
    int64_t t = 0;
    CK(cudaMemcpyAsync(&t, row_ptr + n_a, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *total = t;
    if (t > cap) return fail(ctx, HB_ERR_INVALID_ARG, "pair capacity too small");
    if (t > 0) {
        if (!pairs) return fail(ctx, HB_ERR_INVALID_ARG, "pairs is NULL");
        k1_fill_pairs(a, n_a, b, n_b, n_words, mode, cont_spin, max_degree, lower, row_ptr, pairs, s);
    }
    CK(cudaGetLastError());
    return HB_OK;
}

extern "C" int32_t hb_tuning_report(const hb_ctx *ctx, char *buf, int32_t len) {
    if (!ctx || !buf || len < 1) return -1;
    const std::string r = ctx->plan ? plan_report((const hb::Plan *)ctx->plan) : std::string("no build yet");
    const int32_t n = (int32_t)std::min<size_t>(r.size(), (size_t)len - 1);
    memcpy(buf, r.data(), n);
    buf[n] = 0;
    return (int32_t)r.size();
}

extern "C" int hb_dump(const hb_ctx *ctx, const char *path) {
    if (!ctx || !path) return fail(nullptr, HB_ERR_INVALID_ARG, "NULL argument");
    FILE *f = fopen(path, "w");
    if (!f) return fail(nullptr, HB_ERR_INVALID_ARG, std::string("cannot write ") + path);
    fprintf(f, "orbitals: %d target + %d continuum, n_words %d, electrons %d + 1 (continuum spin %s)\n", ctx->n_to,
            ctx->n_co, ctx->W, ctx->n_elec, ctx->cont_spin == HB_SPIN_ALPHA ? "alpha" : "beta");
    fprintf(f, "dimension %lld = contracted %lld + L2 %d\n", (long long)ctx->dim, (long long)ctx->Dc, ctx->n_l2);
    fprintf(f, "labels K %d (padded %d), e_core %.17g, split slices %d\n", ctx->K, ctx->Kpad, ctx->e_core,
            ctx->split_slices);
    fprintf(f, "expansion panel: %d label class%s of %d columns%s\n", ctx->n_cls, ctx->n_cls > 1 ? "es" : "",
            ctx->Kc, ctx->n_cls > 1 ? " (orbital symmetry)" : "");
    for (int g = 0; g < ctx->n_groups; ++g) {
        const GroupInfo &G = ctx->groups[g];
        fprintf(f, "group %d: %d determinants, %d states, continuum [%d, %d), rows from %lld\n", g, G.ndet, G.ns, G.cf,
                G.cf + G.cn, (long long)G.row_off);
    }
    fprintf(f, "pairs within a double excitation: target x target %lld, target x L2 %lld, L2 x L2 %lld\n",
            (long long)ctx->tt_pairs, (long long)ctx->tl2_pairs, (long long)ctx->l2_nnz);
    fprintf(f, "device bytes %zu, borrows integrals: %s\n", ctx->dev_bytes, ctx->base ? "yes" : "no");
    fprintf(f, "build plan: %s\n", ctx->plan ? plan_report((const hb::Plan *)ctx->plan).c_str() : "no build yet");
    const bool ok = fclose(f) == 0;
    return ok ? HB_OK : fail(nullptr, HB_ERR_INVALID_ARG, std::string("cannot write ") + path);
}

extern "C" const char *hb_last_error(const hb_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_last_error.c_str();
}

void hb::release_lazy(hb_ctx *ctx) {
    if (ctx->plan || ctx->shard_plan) cudaDeviceSynchronize();
    if (ctx->plan) {
        plan_destroy((hb::Plan *)ctx->plan);
        ctx->plan = nullptr;
    }
    if (ctx->shard_plan) {
        plan_destroy((hb::Plan *)ctx->shard_plan);
        ctx->shard_plan = nullptr;
    }
    release_mixed(ctx);
    hb::release_c4tc(ctx);
    hb::release_diag(ctx);
    // the double-float copies (ensure_df) are the allocations after hb_init's
    const size_t n0 = ctx->pool.init_allocs;
    if (ctx->allocs.size() > n0) {
        for (size_t i = n0; i < ctx->allocs.size(); ++i) hb::dfree(ctx, ctx->allocs[i]);
        ctx->allocs.resize(n0);
        ctx->tttc_df = ctx->h_df = ctx->ci_df = ctx->tttt_df = ctx->jk_df = nullptr;
        for (auto &P : ctx->gps) P.A_df = nullptr;
    }
}

extern "C" void hb_destroy(hb_ctx *ctx) {
    if (!ctx) return;
    if (ctx->plan || ctx->shard_plan) cudaDeviceSynchronize();
    if (ctx->plan) {
        plan_destroy((hb::Plan *)ctx->plan);
        ctx->plan = nullptr;
    }
    if (ctx->shard_plan) {
        plan_destroy((hb::Plan *)ctx->shard_plan);
        ctx->shard_plan = nullptr;
    }
    release_mixed(ctx);
    hb::release_c4tc(ctx);
    hb::release_diag(ctx);
    hb::release_mlp(ctx);
    for (void *p : ctx->allocs) hb::dfree(ctx, p);
    delete ctx;
}
