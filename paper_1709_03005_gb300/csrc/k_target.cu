// K2: target-side contraction of the prototype symbols (Eq. 8).
//
// For a pair of target groups (g, g'), with classified determinant pairs
// (m, m') and the CI vectors c, c':
//   S_nn'            = sum_{m m'} c_mn c'_m'n' <D_m|D'_m'>
//   E_nn'            = sum_{m m'} c_mn c'_m'n' <D_m|H^N|D'_m'>
//   gamma^s_nn'(r,q) = sum_{m m'} c_mn c'_m'n' <D_m|a+_{r s} a_{q s}|D'_m'>
// S and E are sparse sandwiches: W = V C' row by row (deterministic order),
// then C^T W by chunked partial sums.  gamma is a sum of phase-weighted outer
// products per key (s, r, q); the contributions are put in key order by a
// stable counting sort so that every sum runs in a fixed order (no floating
// point atomics anywhere).  Every stage is a grouped launch over the group
// pairs of one or many Hamiltonians (one task per group pair).
#include "hb_df.cuh"
#include "hb_tasks.cuh"

namespace hb {

namespace {

// ---------------------------------------------------------------- sandwich
// Wout[m][n'] = sum over records k of row m of v_k * Cp[col_k][n'].  One warp
// per row: lane l takes records l, l+32, ... (fixed order), 16 columns at a
// time, then a butterfly reduction over the lanes (fixed order as well).
// One block per row: warp w of kSWWarps sums the w-th contiguous part of the
// row's records (rows of very different lengths, e.g. a reference determinant
// coupled to every other one, then cost no more than a quarter of the longest),
// each warp reduces by a fixed xor tree and warp 0 adds the warps in order.
constexpr int kSWWarps = 4;

__global__ void __launch_bounds__(32 * kSWWarps)
sandwich_kernel(const SWTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    __shared__ double red[kSWWarps][16];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const SWTask T = tasks[ti];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int row = (int)(blockIdx.x - blk[ti]);
    const int nsp = T.nsp;
    const int64_t b = T.row_ptr[row], e = T.row_ptr[row + 1];
    const int64_t per = (e - b + kSWWarps - 1) / kSWWarps;
    const int64_t kb = b + w * per, ke = min(e, kb + per);
    for (int n0 = 0; n0 < nsp; n0 += 16) {
        double acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = 0.0;
        for (int64_t k = kb + lane; k < ke; k += 32) {
            const int col = T.pairs[k].col;
            const double v = T.val[k];
            const double *crow = T.Cp + (int64_t)col * nsp + n0;
#pragma unroll
            for (int c = 0; c < 16; ++c)
                if (n0 + c < nsp) acc[c] = fma(v, __ldg(crow + c), acc[c]);
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) {
#pragma unroll
            for (int off = 16; off; off >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
        }
        if (lane < 16) {
            double mine = 0.0;
#pragma unroll
            for (int c = 0; c < 16; ++c)
                if (c == lane) mine = acc[c];
            red[w][lane] = mine;
        }
        __syncthreads();
        if (w == 0 && lane < 16 && n0 + lane < nsp) {
            double sum = red[0][lane];
            for (int q = 1; q < kSWWarps; ++q) sum += red[q][lane];
            T.Wout[(int64_t)row * nsp + n0 + lane] = sum;
        }
        __syncthreads();
    }
}

// The same for nsp <= 32: the lanes form G = 32 / P groups of P columns (P the
// power of two >= nsp); group g takes records g, g+G, ... and the groups are
// combined by a butterfly over the lanes that hold the same column.
__global__ void sandwich_small_kernel(const SWTask *__restrict__ tasks, const int64_t *__restrict__ blk,
                                      int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const SWTask T = tasks[ti];
    const int lane = threadIdx.x & 31;
    const int row = (int)(blockIdx.x - blk[ti]) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= T.n_rows) return;
    const int nsp = T.nsp;
    int P = 1;
    while (P < nsp) P <<= 1;
    const int G = 32 / P, g = lane / P, c = lane % P;
    const int64_t b = T.row_ptr[row], e = T.row_ptr[row + 1];
    double acc = 0.0;
    if (c < nsp)
        for (int64_t k = b + g; k < e; k += G) acc = fma(T.val[k], __ldg(T.Cp + (int64_t)T.pairs[k].col * nsp + c), acc);
    for (int off = 16; off >= P; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (g == 0 && c < nsp) T.Wout[(int64_t)row * nsp + c] = acc;
}

// partial[c][n][n'] = sum_{m in chunk c} C[m][n] * Wm[m][n']; rows staged in
// batches, each thread keeps 4 outputs; the task's blocks are (chunk, y) with
// y covering the outputs in steps of 1024.
constexpr int kRowsPerChunk = 256;
// rows (or items) staged per batch so that the staging buffer stays <= 48 KB
__host__ __device__ inline int stage_batch(int ns, int nsp) {
    const int b = 6144 / (ns + nsp);
    return b < 1 ? 1 : (b > 32 ? 32 : b);
}
__global__ void tn_partial_kernel(const TNTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    extern __shared__ double sh[];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const TNTask T = tasks[ti];
    const int lb = (int)(blockIdx.x - blk[ti]);
    const int c = lb / T.ny, by = lb % T.ny;
    const int ns = T.ns, nsp = T.nsp;
    const int kRowBatch = stage_batch(ns, nsp);
    double *cs = sh;                      // [kRowBatch][ns]
    double *ws = sh + kRowBatch * ns;     // [kRowBatch][nsp]
    const int m0 = c * kRowsPerChunk;
    const int rows = min(kRowsPerChunk, T.n_rows - m0);
    const int nout = ns * nsp;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r0 = 0; r0 < rows; r0 += kRowBatch) {
        const int nr = min(kRowBatch, rows - r0);
        __syncthreads();
        for (int i = threadIdx.x; i < nr * ns; i += blockDim.x) cs[i] = T.C[(int64_t)(m0 + r0) * ns + i];
        for (int i = threadIdx.x; i < nr * nsp; i += blockDim.x) ws[i] = T.Wm[(int64_t)(m0 + r0) * nsp + i];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = by * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
            if (t < nout) {
                const int a = t / nsp, b = t % nsp;
                double s = acc[u];
                for (int m = 0; m < nr; ++m) s = fma(cs[m * ns + a], ws[m * nsp + b], s);
                acc[u] = s;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int t = by * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
        if (t < nout) T.partial[(int64_t)c * nout + t] = acc[u];
    }
}

__global__ void reduce_partials_kernel(const TNTask *__restrict__ tasks, const int64_t *__restrict__ blk,
                                       int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const TNTask T = tasks[ti];
    const int t = (int)(blockIdx.x - blk[ti]) * blockDim.x + threadIdx.x;
    const int n_out = T.ns * T.nsp;
    if (t >= n_out) return;
    const int n_chunks = (T.n_rows + kRowsPerChunk - 1) / kRowsPerChunk;
    double acc = 0.0;
    for (int c = 0; c < n_chunks; ++c) acc += T.partial[(int64_t)c * n_out + t];
    T.out[t] = acc;
}

// ------------------------------------------------------------ gamma items
// Per row: number of gamma contributions (deg 0 -> n_elec, deg 1 -> 1).
__global__ void item_count_kernel(const hb_pair *__restrict__ pairs, const int64_t *__restrict__ row_ptr,
                                  int n_rows, int n_elec, int64_t *__restrict__ counts_plus1) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n_rows) return;
    const int64_t b = row_ptr[row], e = row_ptr[row + 1];
    int64_t cnt = 0;
    for (int64_t k = b + lane; k < e; k += 32) {
        const int d = pairs[k].degree;
        cnt += d == 1 ? 1 : 0;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    if (lane == 0) counts_plus1[row + 1] = cnt;
}

// Items in record order, one per single-excitation record.  key = spin *
// n_to^2 + r * n_to + q.  (A deg-0 record is a determinant with itself, m = m'
// of one group; its diagonal contributions gamma(p, p) are the masked C^T C of
// gdiag_partial_kernel below.)
// One block per row: warp w of kIFWarps takes the w-th contiguous part of the
// row's records, counts its items, and writes them after those of the warps
// before it, so the items keep the order of the records.
constexpr int kIFWarps = 4;

__global__ void __launch_bounds__(32 * kIFWarps)
item_fill_kernel(const IFTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    __shared__ int wcnt[kIFWarps];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const IFTask T = tasks[ti];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int row = (int)(blockIdx.x - blk[ti]);
    const int64_t b = T.row_ptr[row], e = T.row_ptr[row + 1];
    const int64_t per = (e - b + kIFWarps - 1) / kIFWarps;
    const int64_t kb = b + w * per, ke = min(e, kb + per);
    int cnt = 0;
    for (int64_t k = kb + lane; k - lane < ke; k += 32) {
        const bool one = k < ke && T.pairs[k].degree == 1;
        cnt += __popc(__ballot_sync(0xffffffffu, one));
    }
    if (lane == 0) wcnt[w] = cnt;
    __syncthreads();
    int64_t pos = T.item_ptr[row];
    for (int q = 0; q < w; ++q) pos += wcnt[q];
    const int W = T.W, n_to = T.n_to;
    const int sb = 64 * W;
    for (int64_t k0 = kb; k0 < ke; k0 += 32) {
        const int64_t k = k0 + lane;
        int one = 0;
        hb_pair r;
        if (k < ke) {
            r = T.pairs[k];
            one = r.degree == 1 ? 1 : 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, one != 0);
        if (one) {
            const int s = r.part[0] / sb, p = r.part[0] % sb, q = r.hole[0] % sb;
            GammaItem it;
            it.key = s * n_to * n_to + p * n_to + q;
            it.m = r.row; it.mp = r.col; it.phase = r.phase;
            T.items[pos + __popc(m & ((1u << lane) - 1u))] = it;
        }
        pos += __popc(m);
    }
}

// --------------------------------------------- diagonal gamma (deg-0 records)
// gamma^s(p, p)[n][n'] over identical determinants (m = m', one group) is
//   sum_{m: p_s occupied in D_m} C[m][n] C[m][n']
// a C^T C with a row mask per spin orbital: chunked partial sums (rows in
// chunks of kRowsPerChunk, fixed order), then a reduction over the chunks.
// Blocks: (chunk, spin orbital sp, y) with y covering the outputs.  A block
// first lists the chunk's rows with p_s occupied (in increasing order, by a
// ballot prefix), then stages only those CI rows.
__host__ __device__ inline int gdiag_batch(int ns) {
    const int b = 5632 / (ns > 0 ? ns : 1);          // 44 KB of staged rows (+ the static row list)
    return b > kRowsPerChunk ? kRowsPerChunk : (b < 1 ? 1 : b);
}

template <bool DF>
__global__ void __launch_bounds__(kRowsPerChunk)
gdiag_partial_kernel(const GDTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    extern __shared__ double gsh[];
    __shared__ int occ_rows[kRowsPerChunk];
    __shared__ int warp_cnt[kRowsPerChunk / 32];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const GDTask T = tasks[ti];
    const int nsp2 = 2 * T.n_to;
    const int lb = (int)(blockIdx.x - blk[ti]);
    const int by = lb % T.ny, sp = (lb / T.ny) % nsp2, c = lb / (T.ny * nsp2);
    const int ns = T.ns, nout = ns * ns;
    const int spin = sp / T.n_to, p = sp % T.n_to;
    const int word = spin * T.W + p / 64;
    const uint64_t bit = 1ull << (p % 64);
    const int m0 = c * kRowsPerChunk;
    const int rows = min(kRowsPerChunk, T.ndet - m0);
    // the chunk's rows with p_s occupied (blockDim.x == kRowsPerChunk)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool o = (int)threadIdx.x < rows && (T.dets[(int64_t)(m0 + threadIdx.x) * 2 * T.W + word] & bit);
    const unsigned bal = __ballot_sync(0xffffffffu, o);
    if (lane == 0) warp_cnt[w] = __popc(bal);
    __syncthreads();
    int pos = __popc(bal & ((1u << lane) - 1u)), n_occ = 0;
    for (int q = 0; q < kRowsPerChunk / 32; ++q) {
        if (q < w) pos += warp_cnt[q];
        n_occ += warp_cnt[q];
    }
    if (o) occ_rows[pos] = threadIdx.x;
    const int kB = gdiag_batch(ns);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    float ah[4] = {0.0f, 0.0f, 0.0f, 0.0f}, al[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int r0 = 0; r0 < n_occ; r0 += kB) {
        const int nr = min(kB, n_occ - r0);
        __syncthreads();
        for (int i = threadIdx.x; i < nr * ns; i += blockDim.x) {
            const int64_t m = m0 + occ_rows[r0 + i / ns];
            if (DF) reinterpret_cast<float2 *>(gsh)[i] = T.C_df[m * ns + i % ns];
            else gsh[i] = T.C[m * ns + i % ns];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = by * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
            if (t < nout) {
                const int a = t / ns, b = t % ns;
                for (int m = 0; m < nr; ++m) {
                    if (DF) {
                        const float2 *cs = reinterpret_cast<const float2 *>(gsh);
                        const float2 x = cs[m * ns + a], y = cs[m * ns + b];
                        df_fma(ah[u], al[u], x.x, x.y, y.x, y.y);
                    } else {
                        acc[u] = fma(gsh[m * ns + a], gsh[m * ns + b], acc[u]);
                    }
                }
            }
        }
    }
    const int64_t base = ((int64_t)c * nsp2 + sp) * nout;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int t = by * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
        if (t < nout) {
            if (DF) reinterpret_cast<float2 *>(T.partial)[base + t] = make_float2(ah[u], al[u]);
            else T.partial[base + t] = acc[u];
        }
    }
}

// gamma[(s, p, p)][t] = sum over the chunks, in order.  Blocks: (sp, t / 256).
template <bool DF>
__global__ void gdiag_reduce_kernel(const GDTask *__restrict__ tasks, const int64_t *__restrict__ blk,
                                    int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const GDTask T = tasks[ti];
    const int nsp2 = 2 * T.n_to, nout = T.ns * T.ns;
    const int tb = (nout + 255) / 256;
    const int lb = (int)(blockIdx.x - blk[ti]);
    const int sp = lb / tb, t = (lb % tb) * 256 + threadIdx.x;
    if (t >= nout) return;
    const int nc = (T.ndet + kRowsPerChunk - 1) / kRowsPerChunk;
    const int spin = sp / T.n_to, p = sp % T.n_to;
    const int64_t key = (int64_t)spin * T.n_to * T.n_to + (int64_t)p * T.n_to + p;
    if (DF) {
        const float2 *part = reinterpret_cast<const float2 *>(T.partial);
        float h = 0.0f, l = 0.0f;
        for (int c = 0; c < nc; ++c) {
            const float2 x = part[((int64_t)c * nsp2 + sp) * nout + t];
            df_add2(h, l, x.x, x.y);
        }
        reinterpret_cast<float2 *>(T.gamma)[key * nout + t] = make_float2(h, l);
    } else {
        double acc = 0.0;
        for (int c = 0; c < nc; ++c) acc += T.partial[((int64_t)c * nsp2 + sp) * nout + t];
        T.gamma[key * nout + t] = acc;
    }
}

// ------------------------------------------------- stable counting sort by key
// Items per chunk of the counting sort: small enough that a short item list
// still spreads over many warps, large enough that the (key, chunk) offset
// table is no larger than the item list (or 2^16 entries).
__host__ __device__ inline int sort_chunk_size(int64_t n_items, int n_keys) {
    int c = 256;
    while (c < 16384 && (n_items + c - 1) / c * (int64_t)n_keys > (n_items > (1 << 16) ? n_items : (1 << 16)))
        c <<= 1;
    return c;
}

__global__ void zero_kernel(const ZTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const ZTask T = tasks[ti];
    const int64_t i0 = (blockIdx.x - blk[ti]) * (int64_t)blockDim.x * 4;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + u * blockDim.x + threadIdx.x;
        if (i < T.n) T.p[i] = 0;
    }
}

// histogram per (key, chunk) in off[1 + key * nc + chunk] (integer atomics: exact)
__global__ void sort_hist_kernel(const SortTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const SortTask T = tasks[ti];
    const int chunk = (int)(blockIdx.x - blk[ti]);
    const int CS = sort_chunk_size(T.n_items, T.n_keys);
    const int64_t base = (int64_t)chunk * CS;
    unsigned long long *hist = (unsigned long long *)T.off;
    for (int i = threadIdx.x; i < CS; i += blockDim.x) {
        const int64_t k = base + i;
        if (k < T.n_items) atomicAdd(hist + 1 + (int64_t)T.items[k].key * T.nc + chunk, 1ull);
    }
}

// Three-phase scan per task over segments of kScanSeg entries:
//   x[0] = 0, x[1..n] := inclusive scan of x[1..n], copy[0..n-1] := x[0..n-1].
// Phase 1: each segment's sum into part[seg]; phase 2 (one block per task):
// exclusive scan of part in place; phase 3: each segment scanned with its
// offset.  Integer sums, so the result is exact in any order.
constexpr int kScanSeg = 4096;

// block-wide inclusive scan of 4 values per thread (1024 threads); returns the
// block total, v[] become inclusive prefixes within the block
__device__ __forceinline__ int64_t block_scan4(int64_t (&v)[4], int64_t *warp_sums) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    v[1] += v[0]; v[2] += v[1]; v[3] += v[2];
    int64_t t = v[3];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, t, off);
        if (lane >= off) t += u;
    }
    if (lane == 31) warp_sums[warp] = t;
    __syncthreads();
    if (warp == 0) {
        int64_t s = warp_sums[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += u;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const int64_t prefix = (warp > 0 ? warp_sums[warp - 1] : 0) + (t - v[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] += prefix;
    const int64_t total = warp_sums[31];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(1024) scan_sums_kernel(const ScanTask *__restrict__ tasks,
                                                         const int64_t *__restrict__ blk, int n_tasks) {
    __shared__ int64_t warp_sums[32];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const ScanTask T = tasks[ti];
    const int64_t seg = blockIdx.x - blk[ti];
    const int64_t i0 = seg * kScanSeg + threadIdx.x * 4;
    int64_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (i0 + k < T.n) ? T.x[1 + i0 + k] : 0;
    const int64_t total = block_scan4(v, warp_sums);
    if (threadIdx.x == 0) T.part[seg] = total;
}

__global__ void __launch_bounds__(1024) scan_part_kernel(const ScanTask *__restrict__ tasks, int n_tasks) {
    __shared__ int64_t warp_sums[32];
    const ScanTask T = tasks[blockIdx.x];
    const int64_t nseg = (T.n + kScanSeg - 1) / kScanSeg;
    int64_t carry = 0;
    for (int64_t base = 0; base < nseg; base += 4096) {
        const int64_t i0 = base + threadIdx.x * 4;
        int64_t v[4], orig[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) orig[k] = v[k] = (i0 + k < nseg) ? T.part[i0 + k] : 0;
        const int64_t total = block_scan4(v, warp_sums);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i0 + k < nseg) T.part[i0 + k] = carry + v[k] - orig[k];     // exclusive
        carry += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) scan_apply_kernel(const ScanTask *__restrict__ tasks,
                                                          const int64_t *__restrict__ blk, int n_tasks) {
    __shared__ int64_t warp_sums[32];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const ScanTask T = tasks[ti];
    const int64_t seg = blockIdx.x - blk[ti];
    const int64_t i0 = seg * kScanSeg + threadIdx.x * 4;
    int64_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (i0 + k < T.n) ? T.x[1 + i0 + k] : 0;
    block_scan4(v, warp_sums);
    const int64_t off = T.part[seg];
    if (seg == 0 && threadIdx.x == 0) {
        T.x[0] = 0;
        if (T.copy && T.n > 0) T.copy[0] = 0;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (i0 + k < T.n) {
            T.x[1 + i0 + k] = v[k] + off;
            if (T.copy && i0 + k + 1 < T.n) T.copy[i0 + k + 1] = v[k] + off;
        }
}

// One warp per chunk walks its items in order, so equal keys keep their order.
// cur: a copy of the exclusive offsets [key][chunk], advanced in place.
__global__ void sort_scatter_kernel(const SortTask *__restrict__ tasks, const int64_t *__restrict__ blk,
                                    int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const SortTask T = tasks[ti];
    const int chunk = (int)(blockIdx.x - blk[ti]);
    const int lane = threadIdx.x;
    const int CS = sort_chunk_size(T.n_items, T.n_keys);
    const int64_t base = (int64_t)chunk * CS;
    for (int i0 = 0; i0 < CS; i0 += 32) {
        const int64_t k = base + i0 + lane;
        const bool valid = k < T.n_items;
        const int key = valid ? T.items[k].key : -1 - lane;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const int leader = __ffs(peers) - 1;
        int64_t *cur = valid ? T.cur + (int64_t)key * T.nc + chunk : nullptr;
        int64_t at = 0;
        if (valid) at = *cur + rank;
        __syncwarp();
        if (valid && lane == leader) *cur += __popc(peers);
        __syncwarp();
        if (valid) T.order[at] = (int32_t)k;
    }
}

// gamma[key][n][n'] = sum over the key's items of phase * C[m][n] * Cp[m'][n']
__global__ void gamma_kernel(const GTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    extern __shared__ double sm[];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const GTask T = tasks[ti];
    const int lb = (int)(blockIdx.x - blk[ti]);
    const int key = lb / T.ny, by = lb % T.ny;
    const int ns = T.ns, nsp = T.nsp;
    const int kItemBatch = stage_batch(ns, nsp);
    double *ca = sm;                          // [kItemBatch][ns]
    double *cb = sm + kItemBatch * ns;        // [kItemBatch][nsp]
    // with no items (nc == 0) both ends are off[0] = 0 and gamma is zero
    const int64_t b = T.off[(int64_t)key * T.nc];
    const int64_t e = T.off[(int64_t)(key + 1) * T.nc];
    if (b == e) return;      // empty key: never written, the coefficient rows read it as zero
    const int nout = ns * nsp;
    // each thread keeps up to 4 outputs in registers
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i0 = b; i0 < e; i0 += kItemBatch) {
        const int cnt = (int)(e - i0 < kItemBatch ? e - i0 : kItemBatch);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt * ns; t += blockDim.x) {
            const int i = t / ns, a = t % ns;
            const GammaItem it = T.items[T.order[i0 + i]];
            ca[i * ns + a] = it.phase * T.C[(int64_t)it.m * ns + a];
        }
        for (int t = threadIdx.x; t < cnt * nsp; t += blockDim.x) {
            const int i = t / nsp, a = t % nsp;
            const GammaItem it = T.items[T.order[i0 + i]];
            cb[i * nsp + a] = T.Cp[(int64_t)it.mp * nsp + a];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = by * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
            if (t < nout) {
                const int a = t / nsp, c = t % nsp;
                double s = acc[u];
                for (int i = 0; i < cnt; ++i) s = fma(ca[i * ns + a], cb[i * nsp + c], s);
                acc[u] = s;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int t = by * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
        if (t < nout) T.gamma[(int64_t)key * nout + t] = acc[u];
    }
}

// The same for small outputs (ns * nsp <= 64): one warp per key, the lanes
// over the outputs, the key's items read in order straight from memory.
__global__ void gamma_warp_kernel(const GTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const GTask T = tasks[ti];
    const int lane = threadIdx.x & 31;
    const int key = (int)(blockIdx.x - blk[ti]) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (key >= T.n_keys) return;
    const int ns = T.ns, nsp = T.nsp, nout = ns * nsp;
    const int64_t b = T.off[(int64_t)key * T.nc];
    const int64_t e = T.off[(int64_t)(key + 1) * T.nc];
    if (b == e) return;
    double acc0 = 0.0, acc1 = 0.0;
    const int t0 = lane, t1 = lane + 32;
    const int a0 = t0 / nsp, c0 = t0 % nsp, a1 = t1 / nsp, c1 = t1 % nsp;
    for (int64_t i = b; i < e; ++i) {
        const GammaItem it = T.items[T.order[i]];
        if (t0 < nout)
            acc0 = fma(it.phase * __ldg(T.C + (int64_t)it.m * ns + a0), __ldg(T.Cp + (int64_t)it.mp * nsp + c0), acc0);
        if (t1 < nout)
            acc1 = fma(it.phase * __ldg(T.C + (int64_t)it.m * ns + a1), __ldg(T.Cp + (int64_t)it.mp * nsp + c1), acc1);
    }
    if (t0 < nout) T.gamma[(int64_t)key * nout + t0] = acc0;
    if (t1 < nout) T.gamma[(int64_t)key * nout + t1] = acc1;
}

// ------------------------------------------------------ coefficient rows
// A[t][k] for the state pairs t = (n, n'):
//   k <  Pt            : Gamma^(r>=s) = sum_spin gamma(r,s) + gamma(s,r) (r != s)
//   Pt <= k < Pt+n_to^2: -gamma^{cont spin}(p, q)
//   k == Pt+n_to^2     : S            (multiplies h_jj')
//   k == Pt+n_to^2+1   : E + e_core S (multiplies delta_jj'); with the target-
//                        energy substitution (Section 3.1) delta_gg' delta_nn' E_n
//   k >= K             : 0
// A key with no items was never written and reads as zero, except the
// diagonal keys of a group with itself (written by the masked C^T C).
// FP64 build: gamma and A in FP64.  Mixed build: gamma as (hi, lo) float
// pairs, the sums in double-float, A written as float pairs (A_df, read by the
// j == j' rows) and as FP64 (read by the slicing).
template <bool DF>
__global__ void assemble_kernel(const ATask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const ATask T = tasks[ti];
    const int t = (int)(blockIdx.x - blk[ti]);
    if (t >= T.n_nn) return;
    const int n = T.nn[2 * t], np = T.nn[2 * t + 1];
    const int ns = T.ns, nsp = T.nsp, n_to = T.n_to, Kpad = T.Kpad;
    const int nout = ns * nsp, sidx = n * nsp + np;
    const int Pt = n_to * (n_to + 1) / 2, nt2 = n_to * n_to;
    auto present = [&](int key, bool diag) -> bool {
        return (diag && T.same) || T.off[(int64_t)key * T.nc] != T.off[(int64_t)(key + 1) * T.nc];
    };
    for (int k = threadIdx.x; k < Kpad; k += blockDim.x) {
        double v = 0.0;
        float vh = 0.0f, vl = 0.0f;
        auto add_key = [&](int key, bool diag, bool neg) {
            if (!present(key, diag)) return;
            if (DF) {
                const float2 g = reinterpret_cast<const float2 *>(T.gamma)[(int64_t)key * nout + sidx];
                df_add2(vh, vl, neg ? -g.x : g.x, neg ? -g.y : g.y);
            } else {
                const double g = T.gamma[(int64_t)key * nout + sidx];
                v += neg ? -g : g;
            }
        };
        if (k < Pt) {
            // unpack k = r(r+1)/2 + s
            int r = (int)((sqrtf(8.0f * (float)k + 1.0f) - 1.0f) * 0.5f);
            while ((r + 1) * (r + 2) / 2 <= k) ++r;
            while (r * (r + 1) / 2 > k) --r;
            const int s = k - r * (r + 1) / 2;
            for (int sp = 0; sp < 2; ++sp) {
                add_key(sp * nt2 + r * n_to + s, r == s, false);
                if (r != s) add_key(sp * nt2 + s * n_to + r, false, false);
            }
        } else if (k < Pt + nt2) {
            const int pq = k - Pt;
            add_key(T.cont_spin * nt2 + pq, pq / n_to == pq % n_to, true);
        } else if (k == Pt + nt2) {
            if (DF) { const float h = (float)T.S[sidx]; vh = h; vl = (float)(T.S[sidx] - (double)h); }
            else v = T.S[sidx];
        } else if (k == Pt + nt2 + 1) {
            const double x = T.En ? ((T.same && n == np && !T.no_En) ? T.En[n] : 0.0)
                                  : T.E[sidx] + T.e_core * T.S[sidx];
            if (DF) { const float h = (float)x; vh = h; vl = (float)(x - (double)h); }
            else v = x;
        }
        if (DF) {
            T.A_df[(int64_t)t * Kpad + k] = make_float2(vh, vl);
            T.A[(int64_t)t * Kpad + k] = df_to_double(vh, vl);
        } else {
            T.A[(int64_t)t * Kpad + k] = v;
        }
    }
}

// ------------------------------------------------ double-float variants
// The same sums on the FP32 pipes for the mixed build: every value is a
// (hi, lo) float pair, products exact by FMA, TwoSum on the high words
// (hb_df.cuh); the order of the terms is the FP64 kernels' order.
__device__ __forceinline__ void shfl_df_add(float &h, float &l, int off) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, off), ol = __shfl_xor_sync(0xffffffffu, l, off);
    df_add2(h, l, oh, ol);
}

// Passes of W states, one block per row as in sandwich_kernel: a lane of warp
// w sums every 32nd record of the warp's part of the row for all W states of
// the pass, the warp reduces by a fixed xor tree and warp 0 adds the warps in
// order.  The coefficient pairs are read 16 bytes at a time where aligned.
template <int W>
__global__ void __launch_bounds__(32 * kSWWarps)
sandwich_df_kernel(const SWTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    __shared__ float2 red[kSWWarps][W];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const SWTask T = tasks[ti];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int row = (int)(blockIdx.x - blk[ti]);
    const int nsp = T.nsp;
    const float2 *val = reinterpret_cast<const float2 *>(T.val);
    float2 *Wout = reinterpret_cast<float2 *>(T.Wout);
    const int64_t b = T.row_ptr[row], e = T.row_ptr[row + 1];
    const int64_t per = (e - b + kSWWarps - 1) / kSWWarps;
    const int64_t kb = b + w * per, ke = min(e, kb + per);
    const bool vec = (nsp & 1) == 0 && (reinterpret_cast<uintptr_t>(T.Cp_df) & 15) == 0;
    for (int n0 = 0; n0 < nsp; n0 += W) {
        float ah[W], al[W];
#pragma unroll
        for (int c = 0; c < W; ++c) { ah[c] = 0.0f; al[c] = 0.0f; }
        for (int64_t k = kb + lane; k < ke; k += 32) {
            const int col = T.pairs[k].col;
            const float2 v = val[k];
            const float2 *crow = T.Cp_df + (int64_t)col * nsp + n0;
            if (vec) {
                // n0 + c even and nsp even: the pair (c, c + 1) is in range together
#pragma unroll
                for (int c = 0; c < W; c += 2)
                    if (n0 + c < nsp) {
                        const float4 x = __ldg(reinterpret_cast<const float4 *>(crow + c));
                        df_fma(ah[c], al[c], v.x, v.y, x.x, x.y);
                        df_fma(ah[c + 1], al[c + 1], v.x, v.y, x.z, x.w);
                    }
            } else {
#pragma unroll
                for (int c = 0; c < W; ++c)
                    if (n0 + c < nsp) {
                        const float2 x = __ldg(crow + c);
                        df_fma(ah[c], al[c], v.x, v.y, x.x, x.y);
                    }
            }
        }
#pragma unroll
        for (int c = 0; c < W; ++c) {
            if (n0 + c < nsp) {
#pragma unroll
                for (int off = 16; off; off >>= 1) shfl_df_add(ah[c], al[c], off);
            }
        }
        if (lane < W) {
            float mh = 0.0f, ml = 0.0f;
#pragma unroll
            for (int c = 0; c < W; ++c)
                if (c == lane) { mh = ah[c]; ml = al[c]; }
            red[w][lane] = make_float2(mh, ml);
        }
        __syncthreads();
        if (w == 0 && lane < W && n0 + lane < nsp) {
            float sh = red[0][lane].x, sl = red[0][lane].y;
            for (int q = 1; q < kSWWarps; ++q) df_add2(sh, sl, red[q][lane].x, red[q][lane].y);
            Wout[(int64_t)row * nsp + n0 + lane] = make_float2(sh, sl);
        }
        __syncthreads();
    }
}

__global__ void sandwich_small_df_kernel(const SWTask *__restrict__ tasks, const int64_t *__restrict__ blk,
                                         int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const SWTask T = tasks[ti];
    const int lane = threadIdx.x & 31;
    const int row = (int)(blockIdx.x - blk[ti]) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= T.n_rows) return;
    const int nsp = T.nsp;
    const float2 *val = reinterpret_cast<const float2 *>(T.val);
    float2 *Wout = reinterpret_cast<float2 *>(T.Wout);
    int P = 1;
    while (P < nsp) P <<= 1;
    const int G = 32 / P, g = lane / P, c = lane % P;
    const int64_t b = T.row_ptr[row], e = T.row_ptr[row + 1];
    // four independent partial sums (records i = 0, 1, 2, 3 mod 4 of this
    // lane's stride), combined in a fixed order
    float h[4] = {0.0f, 0.0f, 0.0f, 0.0f}, l[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (c < nsp) {
        int64_t k = b + g;
        for (; k + 3 * G < e; k += 4 * G) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t kk = k + u * G;
                const float2 v = val[kk];
                const float2 x = __ldg(T.Cp_df + (int64_t)T.pairs[kk].col * nsp + c);
                df_fma(h[u], l[u], v.x, v.y, x.x, x.y);
            }
        }
        for (int u = 0; k < e; k += G, ++u) {
            const float2 v = val[k];
            const float2 x = __ldg(T.Cp_df + (int64_t)T.pairs[k].col * nsp + c);
            df_fma(h[u], l[u], v.x, v.y, x.x, x.y);
        }
    }
    df_add2(h[0], l[0], h[1], l[1]);
    df_add2(h[2], l[2], h[3], l[3]);
    df_add2(h[0], l[0], h[2], l[2]);
    for (int off = 16; off >= P; off >>= 1) shfl_df_add(h[0], l[0], off);
    if (g == 0 && c < nsp) Wout[(int64_t)row * nsp + c] = make_float2(h[0], l[0]);
}

__global__ void tn_partial_df_kernel(const TNTask *__restrict__ tasks, const int64_t *__restrict__ blk,
                                     int n_tasks) {
    extern __shared__ float2 shf[];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const TNTask T = tasks[ti];
    const int lb = (int)(blockIdx.x - blk[ti]);
    const int c = lb / T.ny, by = lb % T.ny;
    const int ns = T.ns, nsp = T.nsp;
    const int kRowBatch = stage_batch(ns, nsp);
    float2 *cs = shf;                     // [kRowBatch][ns]
    float2 *ws = shf + kRowBatch * ns;    // [kRowBatch][nsp]
    const int m0 = c * kRowsPerChunk;
    const int rows = min(kRowsPerChunk, T.n_rows - m0);
    const int nout = ns * nsp;
    float ah[4] = {0.0f, 0.0f, 0.0f, 0.0f}, al[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int r0 = 0; r0 < rows; r0 += kRowBatch) {
        const int nr = min(kRowBatch, rows - r0);
        __syncthreads();
        for (int i = threadIdx.x; i < nr * ns; i += blockDim.x) cs[i] = T.C_df[(int64_t)(m0 + r0) * ns + i];
        for (int i = threadIdx.x; i < nr * nsp; i += blockDim.x) ws[i] = T.Wm_df[(int64_t)(m0 + r0) * nsp + i];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = by * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
            if (t < nout) {
                const int a = t / nsp, b = t % nsp;
                for (int m = 0; m < nr; ++m) {
                    const float2 x = cs[m * ns + a], y = ws[m * nsp + b];
                    df_fma(ah[u], al[u], x.x, x.y, y.x, y.y);
                }
            }
        }
    }
    float2 *partial = reinterpret_cast<float2 *>(T.partial);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int t = by * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
        if (t < nout) partial[(int64_t)c * nout + t] = make_float2(ah[u], al[u]);
    }
}

__global__ void reduce_partials_df_kernel(const TNTask *__restrict__ tasks, const int64_t *__restrict__ blk,
                                          int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const TNTask T = tasks[ti];
    const int t = (int)(blockIdx.x - blk[ti]) * blockDim.x + threadIdx.x;
    const int n_out = T.ns * T.nsp;
    if (t >= n_out) return;
    const int n_chunks = (T.n_rows + kRowsPerChunk - 1) / kRowsPerChunk;
    const float2 *partial = reinterpret_cast<const float2 *>(T.partial);
    float h = 0.0f, l = 0.0f;
    for (int c = 0; c < n_chunks; ++c) {
        const float2 x = partial[(int64_t)c * n_out + t];
        df_add2(h, l, x.x, x.y);
    }
    T.out[t] = df_to_double(h, l);
}

__global__ void gamma_df_kernel(const GTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    extern __shared__ float2 smf[];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const GTask T = tasks[ti];
    const int lb = (int)(blockIdx.x - blk[ti]);
    const int key = lb / T.ny, by = lb % T.ny;
    const int ns = T.ns, nsp = T.nsp;
    const int kItemBatch = stage_batch(ns, nsp);
    float2 *ca = smf;                         // [kItemBatch][ns]
    float2 *cb = smf + kItemBatch * ns;       // [kItemBatch][nsp]
    const int64_t b = T.off[(int64_t)key * T.nc];
    const int64_t e = T.off[(int64_t)(key + 1) * T.nc];
    if (b == e) return;
    const int nout = ns * nsp;
    float ah[4] = {0.0f, 0.0f, 0.0f, 0.0f}, al[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int64_t i0 = b; i0 < e; i0 += kItemBatch) {
        const int cnt = (int)(e - i0 < kItemBatch ? e - i0 : kItemBatch);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt * ns; t += blockDim.x) {
            const int i = t / ns, a = t % ns;
            const GammaItem it = T.items[T.order[i0 + i]];
            float2 x = T.C_df[(int64_t)it.m * ns + a];
            if (it.phase < 0) { x.x = -x.x; x.y = -x.y; }
            ca[i * ns + a] = x;
        }
        for (int t = threadIdx.x; t < cnt * nsp; t += blockDim.x) {
            const int i = t / nsp, a = t % nsp;
            const GammaItem it = T.items[T.order[i0 + i]];
            cb[i * nsp + a] = T.Cp_df[(int64_t)it.mp * nsp + a];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = by * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
            if (t < nout) {
                const int a = t / nsp, c = t % nsp;
                for (int i = 0; i < cnt; ++i) {
                    const float2 x = ca[i * ns + a], y = cb[i * nsp + c];
                    df_fma(ah[u], al[u], x.x, x.y, y.x, y.y);
                }
            }
        }
        // keep the low words small over long keys
#pragma unroll
        for (int u = 0; u < 4; ++u) df_norm(ah[u], al[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int t = by * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
        if (t < nout) reinterpret_cast<float2 *>(T.gamma)[(int64_t)key * nout + t] = make_float2(ah[u], al[u]);
    }
}

__global__ void gamma_warp_df_kernel(const GTask *__restrict__ tasks, const int64_t *__restrict__ blk,
                                     int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const GTask T = tasks[ti];
    const int lane = threadIdx.x & 31;
    const int key = (int)(blockIdx.x - blk[ti]) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (key >= T.n_keys) return;
    const int ns = T.ns, nsp = T.nsp, nout = ns * nsp;
    const int64_t b = T.off[(int64_t)key * T.nc];
    const int64_t e = T.off[(int64_t)(key + 1) * T.nc];
    if (b == e) return;
    float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
    const int t0 = lane, t1 = lane + 32;
    const int a0 = t0 / nsp, c0 = t0 % nsp, a1 = t1 / nsp, c1 = t1 % nsp;
    // renormalise at the block kernel's batch ends, so both forms give the same bits
    const int kb = stage_batch(ns, nsp);
    int since = 0;
    for (int64_t i = b; i < e; ++i) {
        const GammaItem it = T.items[T.order[i]];
        const float sg = it.phase < 0 ? -1.0f : 1.0f;
        if (t0 < nout) {
            const float2 x = __ldg(T.C_df + (int64_t)it.m * ns + a0), y = __ldg(T.Cp_df + (int64_t)it.mp * nsp + c0);
            df_fma(h0, l0, sg * x.x, sg * x.y, y.x, y.y);
        }
        if (t1 < nout) {
            const float2 x = __ldg(T.C_df + (int64_t)it.m * ns + a1), y = __ldg(T.Cp_df + (int64_t)it.mp * nsp + c1);
            df_fma(h1, l1, sg * x.x, sg * x.y, y.x, y.y);
        }
        if (++since == kb || i + 1 == e) {
            since = 0;
            df_norm(h0, l0);
            df_norm(h1, l1);
        }
    }
    float2 *g = reinterpret_cast<float2 *>(T.gamma);
    if (t0 < nout) g[(int64_t)key * nout + t0] = make_float2(h0, l0);
    if (t1 < nout) g[(int64_t)key * nout + t1] = make_float2(h1, l1);
}

}  // namespace

int64_t blocks_rows8(int64_t rows) { return (rows + 7) / 8; }
int tn_chunks(int n_rows) { return (n_rows + kRowsPerChunk - 1) / kRowsPerChunk; }
int tn_ny(int ns, int nsp) { return (ns * nsp + 1023) / 1024; }
int64_t blocks_tn_partial(int n_rows, int ns, int nsp) { return (int64_t)tn_chunks(n_rows) * tn_ny(ns, nsp); }
int64_t blocks_tn_reduce(int ns, int nsp) { return (ns * nsp + 255) / 256; }
int64_t blocks_zero(int64_t n) { return (n + 1023) / 1024; }
int sort_chunks(int64_t n_items, int n_keys) {
    const int c = sort_chunk_size(n_items, n_keys);
    return (int)((n_items + c - 1) / c);
}
int64_t blocks_sort(int64_t n_items, int n_keys) { return sort_chunks(n_items, n_keys); }
int64_t blocks_gamma(int n_keys, int ns, int nsp) { return (int64_t)n_keys * tn_ny(ns, nsp); }
int64_t blocks_gamma_warp(int n_keys) { return (n_keys + 7) / 8; }
size_t smem_stage(int ns, int nsp) { return sizeof(double) * stage_batch(ns, nsp) * (ns + nsp); }

void gamma_item_counts(const hb_pair *pairs, const int64_t *row_ptr, int n_rows, int n_elec,
                       int64_t *counts_plus1, cudaStream_t s) {
    if (n_rows <= 0) return;
    item_count_kernel<<<(n_rows + 7) / 8, 256, 0, s>>>(pairs, row_ptr, n_rows, n_elec, counts_plus1);
}

#define HB_GROUPED(kernel, g, threads, smem, s)                                                     \
    do {                                                                                            \
        if ((g).blocks <= 0) return 0;                                                              \
        kernel<<<(unsigned)(g).blocks, threads, smem, s>>>((g).tasks, (g).blk, (g).n);              \
        return 1;                                                                                   \
    } while (0)

int g_sandwich(const Grouped<SWTask> &g, int dfloat, int width, cudaStream_t s) {
    if (dfloat) {
        if (width <= 16) HB_GROUPED(sandwich_df_kernel<16>, g, 32 * kSWWarps, 0, s);
        if (width <= 24) HB_GROUPED(sandwich_df_kernel<24>, g, 32 * kSWWarps, 0, s);
        HB_GROUPED(sandwich_df_kernel<32>, g, 32 * kSWWarps, 0, s);
    }
    HB_GROUPED(sandwich_kernel, g, 32 * kSWWarps, 0, s);
}
int g_sandwich_small(const Grouped<SWTask> &g, int dfloat, cudaStream_t s) {
    if (dfloat) HB_GROUPED(sandwich_small_df_kernel, g, 256, 0, s);
    HB_GROUPED(sandwich_small_kernel, g, 256, 0, s);
}
int g_tn_partial(const Grouped<TNTask> &g, size_t smem, int dfloat, cudaStream_t s) {
    if (dfloat) HB_GROUPED(tn_partial_df_kernel, g, 256, smem, s);
    HB_GROUPED(tn_partial_kernel, g, 256, smem, s);
}
int g_tn_reduce(const Grouped<TNTask> &g, int dfloat, cudaStream_t s) {
    if (dfloat) HB_GROUPED(reduce_partials_df_kernel, g, 256, 0, s);
    HB_GROUPED(reduce_partials_kernel, g, 256, 0, s);
}
int g_item_fill(const Grouped<IFTask> &g, cudaStream_t s) { HB_GROUPED(item_fill_kernel, g, 32 * kIFWarps, 0, s); }
int g_zero(const Grouped<ZTask> &g, cudaStream_t s) { HB_GROUPED(zero_kernel, g, 256, 0, s); }
int g_sort_hist(const Grouped<SortTask> &g, cudaStream_t s) { HB_GROUPED(sort_hist_kernel, g, 256, 0, s); }
int g_sort_scatter(const Grouped<SortTask> &g, cudaStream_t s) { HB_GROUPED(sort_scatter_kernel, g, 32, 0, s); }
int g_gamma(const Grouped<GTask> &g, size_t smem, int dfloat, cudaStream_t s) {
    if (dfloat) HB_GROUPED(gamma_df_kernel, g, 256, smem, s);
    HB_GROUPED(gamma_kernel, g, 256, smem, s);
}
int g_gamma_warp(const Grouped<GTask> &g, int dfloat, cudaStream_t s) {
    if (dfloat) HB_GROUPED(gamma_warp_df_kernel, g, 256, 0, s);
    HB_GROUPED(gamma_warp_kernel, g, 256, 0, s);
}
int g_assemble(const Grouped<ATask> &g, int dfloat, cudaStream_t s) {
    if (dfloat) HB_GROUPED(assemble_kernel<true>, g, 256, 0, s);
    HB_GROUPED(assemble_kernel<false>, g, 256, 0, s);
}

int g_gdiag(const Grouped<GDTask> &partial, const Grouped<GDTask> &reduce, size_t smem, int dfloat, cudaStream_t s) {
    int L = 0;
    if (partial.blocks > 0) {
        if (dfloat) gdiag_partial_kernel<true><<<(unsigned)partial.blocks, kRowsPerChunk, smem, s>>>(partial.tasks, partial.blk, partial.n);
        else gdiag_partial_kernel<false><<<(unsigned)partial.blocks, kRowsPerChunk, smem, s>>>(partial.tasks, partial.blk, partial.n);
        ++L;
    }
    if (reduce.blocks > 0) {
        if (dfloat) gdiag_reduce_kernel<true><<<(unsigned)reduce.blocks, 256, 0, s>>>(reduce.tasks, reduce.blk, reduce.n);
        else gdiag_reduce_kernel<false><<<(unsigned)reduce.blocks, 256, 0, s>>>(reduce.tasks, reduce.blk, reduce.n);
        ++L;
    }
    return L;
}

int64_t blocks_gdiag_partial(int ndet, int n_to, int ns) {
    return (int64_t)tn_chunks(ndet) * 2 * n_to * tn_ny(ns, ns);
}
int64_t blocks_gdiag_reduce(int n_to, int ns) { return (int64_t)2 * n_to * ((ns * ns + 255) / 256); }
size_t smem_gdiag(int ns) { return sizeof(double) * ns * gdiag_batch(ns); }

int64_t blocks_scan(int64_t n) { return (n + kScanSeg - 1) / kScanSeg; }

int g_scan(const Grouped<ScanTask> &g, cudaStream_t s) {
    if (g.n <= 0) return 0;
    // empty tasks write nothing: their x[0] is zeroed before the histogram
    if (g.blocks <= 0) return 0;
    scan_sums_kernel<<<(unsigned)g.blocks, 1024, 0, s>>>(g.tasks, g.blk, g.n);
    scan_part_kernel<<<g.n, 1024, 0, s>>>(g.tasks, g.n);
    scan_apply_kernel<<<(unsigned)g.blocks, 1024, 0, s>>>(g.tasks, g.blk, g.n);
    return 3;
}

}  // namespace hb
