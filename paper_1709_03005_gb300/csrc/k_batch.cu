// Batched build: many staged Hamiltonians (for instance the spatial-symmetry
// and spin-coupling blocks of one molecule, which share integrals through
// hb_init_shared) built by one CUDA-graph launch.  The build of all of them
// is one plan (k_plan.cu): every stage is a single grouped launch over the
// group pairs of all Hamiltonians, so blocks of very different size fill the
// GPU together, and the short fixed sequence of launches is captured once and
// replayed by hb_batch_launch: the host issues one launch for the whole set.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "hb_api_internal.cuh"
#include "hb_plan.cuh"

struct hb_batch {
    std::vector<hb_ctx *> ctxs;
    std::vector<hb_blocks> outs;
    int precision = HB_FP64;
    hb::Plan *plan = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t nodes = 0;
    int launches = 0;
};

namespace {
thread_local std::string g_batch_error;
int bfail(int code, const std::string &m) {
    g_batch_error = m;
    hb::g_last_error = m;
    return code;
}

void batch_free(hb_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->plan) {
        cudaDeviceSynchronize();
        plan_destroy(b->plan);
    }
    delete b;
}
}  // namespace

extern "C" int hb_batch_create(hb_batch **out, hb_ctx *const *ctxs, int32_t n, int32_t precision,
                               const hb_blocks *outs, void *stream) {
    if (!out || !ctxs || !outs || n < 1) return bfail(HB_ERR_INVALID_ARG, "bad batch arguments");
    if (precision != HB_FP64 && precision != HB_MIXED) return bfail(HB_ERR_INVALID_ARG, "bad precision");
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return bfail(HB_ERR_INVALID_ARG, "NULL context");
    *out = nullptr;
    hb_batch *b = new hb_batch();
    b->precision = precision;
    b->ctxs.assign(ctxs, ctxs + n);
    b->outs.assign(outs, outs + n);
    cudaStream_t s = (cudaStream_t)stream;
    std::string err;
    // the plan prepares the tensor-core operands and uploads its task tables
    int rc = plan_create(ctxs, n, outs, precision, &b->plan, &err, s);
    if (rc != HB_OK) { delete b; return bfail(rc, err); }
    // pick the launch shapes by timing them on this batch's own tasks
    rc = plan_autotune(b->plan, s, &err);
    if (rc != HB_OK) { batch_free(b); return bfail(rc, err); }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { batch_free(b); return bfail(HB_ERR_CUDA, cudaGetErrorString(e)); }
    // capture on a private stream (the legacy default stream cannot be captured)
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { batch_free(b); return bfail(HB_ERR_CUDA, cudaGetErrorString(e)); }
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // the stage events are captured as event-record nodes, so every replay
        // leaves its per-stage times behind
        rc = plan_run(b->plan, cs, true, true, &b->launches, &err);
        cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
        if (rc != HB_OK) rc = bfail(rc, err);
        else if (e2 != cudaSuccess) rc = bfail(HB_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e2));
    } else {
        rc = bfail(HB_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    }
    cudaStreamDestroy(cs);
    if (rc == HB_OK) {
        e = cudaGraphInstantiate(&b->exec, b->graph, cudaGraphInstantiateFlagUseNodePriority);
        if (e != cudaSuccess) rc = bfail(HB_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
        else cudaGraphGetNodes(b->graph, nullptr, &b->nodes);
    }
    if (rc != HB_OK) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return HB_OK;
}

extern "C" int hb_batch_launch(hb_batch *b, hb_stats *st, void *stream) {
    if (!b || !b->exec) return bfail(HB_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
    }
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return bfail(HB_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    if (st) {
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        plan_stats(b->plan, st);
        st->ms_total = ms;
        st->kernel_launches = b->launches;
    }
    if (b->precision == HB_MIXED) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bfail(HB_ERR_CUDA, cudaGetErrorString(e));
        int word = 0;
        if (plan_error_word(b->plan, &word) != HB_OK) return bfail(HB_ERR_CUDA, "reading the mixed error word");
        if (word) return bfail(HB_ERR_TIMEOUT, "a tensor-core kernel gave up waiting (code " + std::to_string(word) + ")");
    }
    return HB_OK;
}

extern "C" int hb_batch_nodes(const hb_batch *b) { return b ? (int)b->nodes : -1; }

extern "C" int32_t hb_batch_report(const hb_batch *b, char *buf, int32_t len) {
    if (!b || !buf || len < 1) return -1;
    const std::string r = plan_report(b->plan);
    const int32_t n = (int32_t)std::min<size_t>(r.size(), (size_t)len - 1);
    memcpy(buf, r.data(), n);
    buf[n] = 0;
    return (int32_t)r.size();
}

extern "C" void hb_batch_destroy(hb_batch *b) {
    if (!b) return;
    batch_free(b);
}
