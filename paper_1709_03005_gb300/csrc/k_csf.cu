// Spin-adapted target groups (configuration state functions) and groups that
// share their determinants.
//
// A target state of Eq. 2 is phi_n = sum_i c_in eta_i with eta_i a CSF, itself
// a fixed combination of determinants, eta_i = sum_d b_id D_d.  The build works
// on determinants, so its CI vectors are C[d][n] = sum_i b_id c_in: one more
// contraction level ahead of the prototype contraction of Eq. 8, done here on
// the device, one thread per (determinant, state), the terms of a determinant
// summed in CSF order.
//
// Groups whose determinant sets are equal (a singlet and a triplet target over
// the same configurations, coupled to the same continuum) are built as one
// group whose states are the groups' states in order: its rows (state-major,
// then continuum orbital) are the groups' rows one after the other, so the
// layout of the result does not change, and every coupling between the two
// spin states (overlap, H^N and transition densities over shared
// determinants) is computed by the same-group path.
#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "hb_api_internal.cuh"

namespace hb {

namespace {

__global__ void csf_expand_kernel(const int64_t *__restrict__ dptr, const int32_t *__restrict__ dcsf,
                                  const double *__restrict__ dcoef, int n_det, const double *__restrict__ ci_csf,
                                  int ns, double *__restrict__ C, int ld, int col_off) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_det * ns) return;
    const int d = (int)(t / ns), n = (int)(t % ns);
    double acc = 0.0;
    for (int64_t k = dptr[d]; k < dptr[d + 1]; ++k) acc = fma(dcoef[k], ci_csf[(int64_t)dcsf[k] * ns + n], acc);
    C[(int64_t)d * ld + col_off + n] = acc;
}

bool same_det_set(const hb_group &a, const hb_group &b, int nw) {
    if (a.n_det != b.n_det) return false;
    std::vector<std::vector<uint64_t>> x, y;
    for (int m = 0; m < a.n_det; ++m) {
        x.emplace_back(a.dets + (size_t)m * nw, a.dets + (size_t)(m + 1) * nw);
        y.emplace_back(b.dets + (size_t)m * nw, b.dets + (size_t)(m + 1) * nw);
    }
    std::sort(x.begin(), x.end());
    std::sort(y.begin(), y.end());
    return x == y;
}

}  // namespace

int prepare_groups(const hb_problem *p, GroupPlan *out, std::string *err) {
    out->needed = false;
    if (!p || p->n_groups <= 0 || !p->groups) return HB_OK;
    const int nw = 2 * p->n_words;
    for (int g = 0; g < p->n_groups; ++g) {
        const hb_group &G = p->groups[g];
        if (G.n_csf != 0) out->needed = true;
        if (g > 0 && G.n_det == p->groups[g - 1].n_det && G.cont_first == p->groups[g - 1].cont_first &&
            G.cont_count == p->groups[g - 1].cont_count && G.dets && p->groups[g - 1].dets &&
            same_det_set(G, p->groups[g - 1], nw))
            out->needed = true;
    }
    if (!out->needed) return HB_OK;
    // members of each merged group: runs of adjacent groups with the same
    // determinant set and continuum range
    std::vector<std::vector<int>> runs;
    for (int g = 0; g < p->n_groups; ++g) {
        const hb_group &G = p->groups[g];
        if (G.n_det < 1 || G.n_state < 1 || !G.dets || !G.ci) {
            *err = "group " + std::to_string(g) + ": empty or NULL";
            return HB_ERR_INVALID_ARG;
        }
        bool join = false;
        if (!runs.empty()) {
            const hb_group &F = p->groups[runs.back().front()];
            join = G.cont_first == F.cont_first && G.cont_count == F.cont_count && same_det_set(G, F, nw);
        }
        if (join) runs.back().push_back(g);
        else runs.push_back({g});
    }
    const bool energies = p->groups[0].energy != nullptr;
    out->groups.clear();
    out->members.clear();
    out->zero_ci.assign(runs.size(), {});
    out->energy.assign(runs.size(), {});
    out->user_of.assign(p->n_groups, {0, 0});
    for (size_t r = 0; r < runs.size(); ++r) {
        const hb_group &F = p->groups[runs[r].front()];
        // the merged group's determinant order is the first member's
        std::map<std::vector<uint64_t>, int> pos;
        for (int m = 0; m < F.n_det; ++m) pos[std::vector<uint64_t>(F.dets + (size_t)m * nw, F.dets + (size_t)(m + 1) * nw)] = m;
        int ns_tot = 0;
        for (int g : runs[r]) {
            const hb_group &G = p->groups[g];
            GroupPlan::Member M;
            M.internal = (int)r;
            M.col_off = ns_tot;
            M.ns = G.n_state;
            M.ci = G.ci;
            out->user_of[g] = {(int)r, ns_tot};
            // determinant -> (CSF, coefficient) lists, in the merged order
            std::vector<std::vector<std::pair<int32_t, double>>> per(F.n_det);
            std::vector<int> map(G.n_det);
            for (int m = 0; m < G.n_det; ++m)
                map[m] = pos.at(std::vector<uint64_t>(G.dets + (size_t)m * nw, G.dets + (size_t)(m + 1) * nw));
            if (G.n_csf > 0) {
                if (!G.csf_ptr || !G.csf_det || !G.csf_coef || G.csf_ptr[0] != 0) {
                    *err = "group " + std::to_string(g) + ": CSF arrays NULL or csf_ptr[0] != 0";
                    return HB_ERR_INVALID_ARG;
                }
                for (int i = 0; i < G.n_csf; ++i) {
                    if (G.csf_ptr[i + 1] < G.csf_ptr[i]) {
                        *err = "group " + std::to_string(g) + ": csf_ptr decreases";
                        return HB_ERR_INVALID_ARG;
                    }
                    for (int k = G.csf_ptr[i]; k < G.csf_ptr[i + 1]; ++k) {
                        const int d = G.csf_det[k];
                        if (d < 0 || d >= G.n_det || !std::isfinite(G.csf_coef[k])) {
                            *err = "group " + std::to_string(g) + ": CSF determinant index or coefficient";
                            return HB_ERR_INVALID_ARG;
                        }
                        per[map[d]].push_back({(int32_t)i, G.csf_coef[k]});
                    }
                }
                M.n_csf = G.n_csf;
            } else {
                for (int m = 0; m < G.n_det; ++m) per[map[m]].push_back({(int32_t)m, 1.0});
                M.n_csf = G.n_det;
            }
            for (size_t i = 0; i < (size_t)M.n_csf * M.ns; ++i)
                if (!std::isfinite(G.ci[i])) {
                    *err = "group " + std::to_string(g) + ": non-finite CI";
                    return HB_ERR_INVALID_ARG;
                }
            M.dptr.assign(1, 0);
            for (auto &v : per) {
                std::stable_sort(v.begin(), v.end(), [](auto &a, auto &b) { return a.first < b.first; });
                for (auto &e : v) {
                    M.dcsf.push_back(e.first);
                    M.dcoef.push_back(e.second);
                }
                M.dptr.push_back((int64_t)M.dcsf.size());
            }
            if (energies && G.energy)
                out->energy[r].insert(out->energy[r].end(), G.energy, G.energy + G.n_state);
            ns_tot += G.n_state;
            out->members.push_back(std::move(M));
        }
        hb_group I = F;
        I.n_state = ns_tot;
        out->zero_ci[r].assign((size_t)F.n_det * ns_tot, 0.0);
        I.ci = out->zero_ci[r].data();
        I.energy = energies ? out->energy[r].data() : nullptr;
        I.n_csf = 0;
        I.csf_ptr = nullptr;
        I.csf_det = nullptr;
        I.csf_coef = nullptr;
        out->groups.push_back(I);
    }
    return HB_OK;
}

int expand_group_ci(hb_ctx *ctx, const GroupPlan &plan, cudaStream_t s, std::string *err) {
    for (const auto &M : plan.members) {
        const GroupInfo &gi = ctx->groups[M.internal];
        int64_t *dptr = nullptr;
        int32_t *dcsf = nullptr;
        double *dcoef = nullptr, *ci = nullptr;
        const size_t nnz = std::max<size_t>(M.dcsf.size(), 1);
        cudaError_t e = cudaMalloc(&dptr, sizeof(int64_t) * M.dptr.size());
        if (e == cudaSuccess) e = cudaMalloc(&dcsf, sizeof(int32_t) * nnz);
        if (e == cudaSuccess) e = cudaMalloc(&dcoef, sizeof(double) * nnz);
        if (e == cudaSuccess) e = cudaMalloc(&ci, sizeof(double) * std::max<size_t>((size_t)M.n_csf * M.ns, 1));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dptr, M.dptr.data(), sizeof(int64_t) * M.dptr.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !M.dcsf.empty())
            e = cudaMemcpyAsync(dcsf, M.dcsf.data(), sizeof(int32_t) * M.dcsf.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !M.dcoef.empty())
            e = cudaMemcpyAsync(dcoef, M.dcoef.data(), sizeof(double) * M.dcoef.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ci, M.ci, sizeof(double) * (size_t)M.n_csf * M.ns, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            const int64_t n = (int64_t)gi.ndet * M.ns;
            csf_expand_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dptr, dcsf, dcoef, gi.ndet, ci, M.ns,
                                                                         ctx->ci + gi.ci_off, gi.ns, M.col_off);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(dptr);
        cudaFree(dcsf);
        cudaFree(dcoef);
        cudaFree(ci);
        if (e != cudaSuccess) {
            *err = std::string("CSF expansion: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? HB_ERR_OOM : HB_ERR_CUDA;
        }
    }
    return HB_OK;
}

}  // namespace hb
