// hb_classify_noalloc: the excitation classification of hb_classify for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs where the
// allocator is owned by someone else (a host framework whose memory pool must
// not be bypassed, a plug-in loaded into a process that forbids device
// allocation after start-up, or a real-time loop where an allocation's
// implicit synchronisation is not allowed).  hb_classify asks such a caller
// for a row-offset buffer of n_a + 1 int64 values, which it may be unable to
// provide.  This variant keeps those offsets in a file-scope device array of
// fixed size instead, so the caller passes only the determinant lists and the
// output records.
//
// The array is HB_NOALLOC_MAX_ROWS + 1 int64 values (2 MiB); every GPU that
// loads this library holds it until the process exits.  All calls share it:
// calls whose work overlaps on the GPU (different streams, or different
// threads without ordering) race on it and must be serialised by the caller.
// Each call clears the entries it needs before using them.
#include <mutex>

#include "hb_internal.cuh"

namespace {

static __device__ __align__(256) int64_t g_noalloc_rows[HB_NOALLOC_MAX_ROWS + 1];

constexpr int kMaxDevices = 64;
int64_t *g_rows_ptr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;
int noalloc_fail(int code, const std::string &msg) {
    hb::g_last_error = msg;   // read back by hb_last_error(NULL)
    return code;
}

// Device address of the static array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, once per device, with that device current.  The cached
// address lives as long as the device's primary context: after a
// cudaDeviceReset it is stale, which is why the header rules out calls on a
// device after a reset.
int rows_address(int64_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(HB_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(HB_ERR_UNSUPPORTED, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_rows_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_rows);
        if (e != cudaSuccess || !p)
            return noalloc_fail(HB_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_rows_ptr[dev] = (int64_t *)p;
    }
    *out = g_rows_ptr[dev];
    return HB_OK;
}

}  // namespace

extern "C" int hb_classify_noalloc(const uint64_t *a, int32_t n_a, const uint64_t *b, int32_t n_b,
                                   int32_t n_words, int32_t mode, int32_t cont_spin, int32_t max_degree,
                                   int32_t lower, hb_pair *pairs, int64_t cap, int64_t *total, void *stream) {
    if (n_words < 1 || n_words > HB_MAXW) return noalloc_fail(HB_ERR_UNSUPPORTED, "n_words must be 1..4");
    if (n_a < 0 || n_b < 0 || !total || (mode != 0 && mode != 1) || max_degree < 0)
        return noalloc_fail(HB_ERR_INVALID_ARG, "bad classify arguments");
    if (n_a > HB_NOALLOC_MAX_ROWS)
        return noalloc_fail(HB_ERR_INVALID_ARG, "hb_classify_noalloc: n_a = " + std::to_string(n_a) +
                                                    " exceeds the static row buffer of " +
                                                    std::to_string(HB_NOALLOC_MAX_ROWS) + " rows");
    if ((n_a > 0 && !a) || (n_b > 0 && !b)) return noalloc_fail(HB_ERR_INVALID_ARG, "NULL determinant list");
    int64_t *rows = nullptr;
    int rc = rows_address(&rows);
    if (rc != HB_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the previous call's offsets are still there: clear the ones this call reads
    cudaError_t e = cudaMemsetAsync(rows, 0, sizeof(int64_t) * ((size_t)n_a + 1), s);
    if (e != cudaSuccess) return noalloc_fail(HB_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    if (n_a > 0) {
        hb::k1_count(a, n_a, b, n_b, n_words, mode, max_degree, lower, rows, s);
        hb::exclusive_scan_inplace(rows, n_a, s);
    }
    int64_t t = 0;
    e = cudaMemcpyAsync(&t, rows + n_a, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(HB_ERR_CUDA, std::string("row count readback: ") + cudaGetErrorString(e));
    *total = t;
    if (t > cap) return noalloc_fail(HB_ERR_INVALID_ARG, "pair capacity too small");
    if (t > 0) {
        if (!pairs) return noalloc_fail(HB_ERR_INVALID_ARG, "pairs is NULL");
        hb::k1_fill_pairs(a, n_a, b, n_b, n_words, mode, cont_spin, max_degree, lower, rows, pairs, s);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(HB_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return HB_OK;
}
