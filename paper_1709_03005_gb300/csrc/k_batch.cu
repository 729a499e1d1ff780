// Batched build: many staged Hamiltonians (for instance the spatial-symmetry
// and spin-coupling blocks of one molecule, which share integrals through
// hb_init_shared) built by one CUDA-graph launch.  The graph is captured once
// from the ordinary build of every context (after one eager build that sets up
// the tensor-core operands), each context on its own branch so that their
// kernels overlap, and replayed by hb_batch_launch: the host issues a single
// launch for the whole set of uneven blocks.
#include <cstring>
#include <string>
#include <vector>

#include "hb_api_internal.cuh"

struct hb_batch {
    std::vector<hb_ctx *> ctxs;
    std::vector<hb_blocks> outs;
    int precision = HB_FP64;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t nodes = 0;
};

namespace {
thread_local std::string g_batch_error;
int bfail(int code, const std::string &m) {
    g_batch_error = m;
    hb::g_last_error = m;
    return code;
}
}  // namespace

extern "C" int hb_batch_create(hb_batch **out, hb_ctx *const *ctxs, int32_t n, int32_t precision,
                               const hb_blocks *outs, void *stream) {
    if (!out || !ctxs || !outs || n < 1) return bfail(HB_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    hb_batch *b = new hb_batch();
    b->precision = precision;
    b->ctxs.assign(ctxs, ctxs + n);
    b->outs.assign(outs, outs + n);
    cudaStream_t s = (cudaStream_t)stream;
    // eager build: allocates and slices the tensor-core operands, sets kernel attributes
    for (int i = 0; i < n; ++i) {
        int rc = hb_build_blocks(ctxs[i], precision, &outs[i], nullptr, s);
        if (rc != HB_OK) { delete b; return bfail(rc, std::string("eager build: ") + hb_last_error(ctxs[i])); }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { delete b; return bfail(HB_ERR_CUDA, cudaGetErrorString(e)); }
    // capture on a private stream (the legacy default stream cannot be captured);
    // every context is its own branch of the graph (fork / join through events),
    // so the small kernels of different Hamiltonians run concurrently
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete b; return bfail(HB_ERR_CUDA, cudaGetErrorString(e)); }
    std::vector<cudaStream_t> br(n, nullptr);
    std::vector<cudaEvent_t> done(n, nullptr);
    cudaEvent_t fork = nullptr;
    cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int i = 0; i < n; ++i) {
        cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming);
    }
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = HB_OK;
    if (e == cudaSuccess) {
        cudaEventRecord(fork, cs);
        for (int i = 0; i < n && rc == HB_OK; ++i) {
            cudaStreamWaitEvent(br[i], fork, 0);
            ctxs[i]->capturing = true;
            rc = hb_build_blocks(ctxs[i], precision, &outs[i], nullptr, br[i]);
            ctxs[i]->capturing = false;
            cudaEventRecord(done[i], br[i]);
            cudaStreamWaitEvent(cs, done[i], 0);
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
        if (e2 != cudaSuccess && rc == HB_OK) rc = bfail(HB_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e2));
    } else {
        rc = bfail(HB_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    }
    for (int i = 0; i < n; ++i) {
        cudaStreamDestroy(br[i]);
        cudaEventDestroy(done[i]);
    }
    cudaEventDestroy(fork);
    cudaStreamDestroy(cs);
    if (rc == HB_OK) {
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) rc = bfail(HB_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
        cudaGraphGetNodes(b->graph, nullptr, &b->nodes);
    }
    if (rc != HB_OK) {
        if (b->graph) cudaGraphDestroy(b->graph);
        delete b;
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
        memset(st, 0, sizeof(*st));
        st->ms_total = ms;
        st->kernel_launches = (int32_t)b->nodes;
    }
    if (b->precision == HB_MIXED) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bfail(HB_ERR_CUDA, cudaGetErrorString(e));
        for (hb_ctx *c : b->ctxs) {
            int word = 0;
            if (mixed_error_word(c, &word) != HB_OK) return bfail(HB_ERR_CUDA, "reading the mixed error word");
            if (word) return bfail(HB_ERR_TIMEOUT, "split expansion kernel gave up waiting");
        }
    }
    return HB_OK;
}

extern "C" int hb_batch_nodes(const hb_batch *b) { return b ? (int)b->nodes : -1; }

extern "C" void hb_batch_destroy(hb_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}
