// K1: excitation classification of determinant pairs (Section 2.1).
//
// One warp per row determinant; the 32 lanes take 32 consecutive column
// determinants at a time (coalesced 16*W-byte loads), compute the excitation
// degree with XOR + popcount, and compact the pairs within a double excitation
// with a ballot, so the output is ordered by (row, col) without atomics.
// Holes and particles come from the set bits of (ket & ~bra) and (bra & ~ket);
// the phase comes from prefix popcounts of the ket string (the sign of applying
// the annihilation and creation operators one after the other).
#include "hb_tasks.cuh"

namespace hb {

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kSeg = kSegCols;   // columns per segment of the hot scans

template <int W>
__device__ __forceinline__ void load_det(const uint64_t *p, uint64_t (&x)[2 * W]) {
#pragma unroll
    for (int i = 0; i < 2 * W; ++i) x[i] = __ldg(p + i);
}

// mode 0: degree = popc(a ^ b) / 2.  mode 1: a is an (N+1)-electron L2
// determinant, b an N-electron target determinant that gets one continuum
// electron; degree = popc(b & ~a) + 1.
template <int W, int MODE>
__device__ __forceinline__ int degree_of(const uint64_t (&a)[2 * W], const uint64_t (&b)[2 * W]) {
    int c = 0;
#pragma unroll
    for (int i = 0; i < 2 * W; ++i) c += MODE == 0 ? __popcll(a[i] ^ b[i]) : __popcll(b[i] & ~a[i]);
    return MODE == 0 ? (c >> 1) : c + 1;
}

// Up to two set-bit positions of (x & ~y), ascending.
template <int W>
__device__ __forceinline__ int bits_of_diff(const uint64_t (&x)[2 * W], const uint64_t (&y)[2 * W],
                                            int (&pos)[2]) {
    int n = 0;
#pragma unroll
    for (int i = 0; i < 2 * W; ++i) {
        uint64_t m = x[i] & ~y[i];
        while (m && n < 2) {
            pos[n++] = 64 * i + (__ffsll((long long)m) - 1);
            m &= m - 1;
        }
    }
    return n;
}

// Sign exponent of <bra| a+_p1 a+_p2 a_h2 a_h1 |ket> for holes h1<h2 and
// particles p1<p2 (keys in canonical order), ck(x) = # ket electrons below x.
__device__ __forceinline__ int double_exponent(int ch1, int ch2, int cp1, int cp2, int kh1, int kh2,
                                               int kp1, int kp2) {
    return ch1 + ch2 - 1 + cp2 - (kh1 < kp2) - (kh2 < kp2) + cp1 - (kh1 < kp1) - (kh2 < kp1);
}

template <int W, int MODE>
__device__ __forceinline__ void make_record(const uint64_t (&a)[2 * W], const uint64_t (&b)[2 * W],
                                            int deg, int cont_spin, int row, int col, hb_pair &r) {
    r.row = row;
    r.col = col;
    r.degree = (int8_t)deg;
    r.hole[0] = r.hole[1] = r.part[0] = r.part[1] = -1;
    r.pad[0] = r.pad[1] = r.pad[2] = 0;
    int e = 0;
    if (MODE == 0) {
        // bra = a (row), ket = b (col)
        int h[2], p[2];
        bits_of_diff<W>(b, a, h);
        bits_of_diff<W>(a, b, p);
        if (deg == 1) {
            e = prefix_count(b, 2 * W, h[0]) + prefix_count(b, 2 * W, p[0]) - (h[0] < p[0]);
            r.hole[0] = (int16_t)h[0];
            r.part[0] = (int16_t)p[0];
        } else if (deg == 2) {
            e = double_exponent(prefix_count(b, 2 * W, h[0]), prefix_count(b, 2 * W, h[1]),
                                prefix_count(b, 2 * W, p[0]), prefix_count(b, 2 * W, p[1]), h[0], h[1],
                                p[0], p[1]);
            r.hole[0] = (int16_t)h[0]; r.hole[1] = (int16_t)h[1];
            r.part[0] = (int16_t)p[0]; r.part[1] = (int16_t)p[1];
        }
    } else {
        // bra = b + continuum electron v (spin cont_spin), ket = a (row).
        // Keys are doubled bit positions; v sits just above the last target
        // orbital of its spin.
        const int kv = cont_spin == 0 ? 2 * 64 * W - 1 : 2 * 128 * W - 1;
        const int cv = cont_spin == 0 ? prefix_count(a, 2 * W, 64 * W) : prefix_count(a, 2 * W, 128 * W);
        int h[2], q[2];
        const int nh = bits_of_diff<W>(a, b, h);   // in chi only: d + 1
        const int nq = bits_of_diff<W>(b, a, q);   // in D only: d
        if (deg == 1 && nh >= 1) {
            const int kh = 2 * h[0];
            e = prefix_count(a, 2 * W, h[0]) + cv - (kh < kv);
            r.hole[0] = (int16_t)h[0];
        } else if (deg == 2 && nh == 2 && nq == 1) {
            const int kq = 2 * q[0];
            int kp1, kp2, cp1, cp2;
            const int cq = prefix_count(a, 2 * W, q[0]);
            if (kq < kv) { kp1 = kq; cp1 = cq; kp2 = kv; cp2 = cv; }
            else { kp1 = kv; cp1 = cv; kp2 = kq; cp2 = cq; }
            e = double_exponent(prefix_count(a, 2 * W, h[0]), prefix_count(a, 2 * W, h[1]), cp1, cp2,
                                2 * h[0], 2 * h[1], kp1, kp2);
            r.hole[0] = (int16_t)h[0]; r.hole[1] = (int16_t)h[1];
            r.part[0] = (int16_t)q[0];
        }
    }
    r.phase = (e & 1) ? (int8_t)-1 : (int8_t)1;
}

template <int W, int MODE>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
k1_count_kernel(const uint64_t *__restrict__ A, int n_a, const uint64_t *__restrict__ B, int n_b,
                int max_degree, int lower, int64_t *__restrict__ counts_plus1) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (row >= n_a) return;
    uint64_t a[2 * W];
    load_det<W>(A + (int64_t)row * 2 * W, a);
    const int limit = lower ? min(n_b, row + 1) : n_b;
    int cnt = 0;
    for (int c0 = 0; c0 < limit; c0 += 32) {
        const int c = c0 + lane;
        bool ok = false;
        if (c < limit) {
            uint64_t b[2 * W];
            load_det<W>(B + (int64_t)c * 2 * W, b);
            ok = degree_of<W, MODE>(a, b) <= max_degree;
        }
        cnt += __popc(__ballot_sync(0xffffffffu, ok));
    }
    if (lane == 0) counts_plus1[row + 1] = cnt;
}

// Matches of each row within each segment of kSeg columns (one warp per
// (row, segment)), turned into offsets from the row start by seg_scan_kernel.
template <int W, int MODE>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
k1_seg_count_kernel(const uint64_t *__restrict__ A, int n_a, const uint64_t *__restrict__ B, int n_b,
                    int max_degree, int lower, int nseg, int32_t *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (wid >= (int64_t)n_a * nseg) return;
    const int row = (int)(wid / nseg), sg = (int)(wid % nseg);
    uint64_t a[2 * W];
    load_det<W>(A + (int64_t)row * 2 * W, a);
    const int limit = lower ? min(n_b, row + 1) : n_b;
    const int c_end = min(limit, (sg + 1) * kSeg);
    int c_cnt = 0;
    for (int c0 = sg * kSeg; c0 < c_end; c0 += 32) {
        const int c = c0 + lane;
        bool ok = false;
        if (c < c_end) {
            uint64_t b[2 * W];
            load_det<W>(B + (int64_t)c * 2 * W, b);
            ok = degree_of<W, MODE>(a, b) <= max_degree;
        }
        c_cnt += __popc(__ballot_sync(0xffffffffu, ok));
    }
    if (lane == 0) cnt[wid] = c_cnt;
}

__global__ void seg_scan_kernel(int32_t *__restrict__ cnt, int n_a, int nseg) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n_a) return;
    int32_t acc = 0;
    for (int sg = 0; sg < nseg; ++sg) {
        const int32_t c = cnt[(int64_t)row * nseg + sg];
        cnt[(int64_t)row * nseg + sg] = acc;
        acc += c;
    }
}

template <int W, int MODE>
__device__ __forceinline__ void fill_row(const uint64_t *__restrict__ A, const uint64_t *__restrict__ B, int n_b,
                                         int cont_spin, int max_degree, int lower,
                                         const int64_t *__restrict__ row_ptr, hb_pair *__restrict__ out, int row,
                                         int lane) {
    uint64_t a[2 * W];
    load_det<W>(A + (int64_t)row * 2 * W, a);
    const int limit = lower ? min(n_b, row + 1) : n_b;
    int64_t pos = row_ptr[row];
    const int64_t end = row_ptr[row + 1];
    for (int c0 = 0; c0 < limit; c0 += 32) {
        const int c = c0 + lane;
        bool ok = false;
        int deg = 99;
        uint64_t b[2 * W];
        if (c < limit) {
            load_det<W>(B + (int64_t)c * 2 * W, b);
            deg = degree_of<W, MODE>(a, b);
            ok = deg <= max_degree;
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const int64_t at = pos + __popc(m & ((1u << lane) - 1u));
            if (at < end) {
                hb_pair r;
                make_record<W, MODE>(a, b, deg, cont_spin, row, c, r);
                out[at] = r;
            }
        }
        pos += __popc(m);
    }
}

template <int W, int MODE>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
k1_fill_kernel(const uint64_t *__restrict__ A, int n_a, const uint64_t *__restrict__ B, int n_b,
               int cont_spin, int max_degree, int lower, const int64_t *__restrict__ row_ptr,
               hb_pair *__restrict__ out) {
    const int row = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (row >= n_a) return;
    fill_row<W, MODE>(A, B, n_b, cont_spin, max_degree, lower, row_ptr, out, row, threadIdx.x & 31);
}

// The same over many (a, b) tasks in one launch, with the column
// determinants staged through shared memory: the 8 warps of a block (8 rows)
// read each tile of columns from memory once, word-major so the lanes'
// shared-memory reads are conflict free.
template <int W>
struct ColTile {
    static constexpr int kCols = kSeg;       // a segment of column determinants
};

template <int W>
__device__ __forceinline__ void stage_cols(uint64_t *tile, const uint64_t *__restrict__ B, int t0, int tn) {
    constexpr int TC = ColTile<W>::kCols;
    for (int i = threadIdx.x; i < tn * 2 * W; i += blockDim.x) {
        const int c = i / (2 * W), w = i % (2 * W);
        tile[w * TC + c] = __ldg(B + (int64_t)t0 * 2 * W + i);
    }
}

template <int W>
__device__ __forceinline__ void tile_det(const uint64_t *tile, int c, uint64_t (&b)[2 * W]) {
#pragma unroll
    for (int w = 0; w < 2 * W; ++w) b[w] = tile[w * ColTile<W>::kCols + c];
}

// Matches are queued per warp (in column order) and turned into records 32
// at a time, one per lane, so the record work never runs with a lone lane.
template <int W, int MODE>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
k1_fill_grouped(const ClsTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    constexpr int TC = ColTile<W>::kCols;
    __shared__ uint64_t tile[TC * 2 * W];
    __shared__ int queue[kWarpsPerBlock][64];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const ClsTask &T = tasks[ti];
    const int lb = (int)(blockIdx.x - blk[ti]);
    // block = (8 rows, one segment of columns)
    const int rb = lb / T.nseg, sg = lb % T.nseg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row = rb * kWarpsPerBlock + warp;
    const bool active = row < T.n_a;
    int *q = queue[warp];
    uint64_t a[2 * W];
    int limit = 0;
    int64_t pos = 0, end = 0;
    if (active) {
        load_det<W>(T.a + (int64_t)row * 2 * W, a);
        limit = T.lower ? min(T.n_b, row + 1) : T.n_b;
        pos = T.row_ptr[row] + T.seg_off[(int64_t)row * T.nseg + sg];
        end = T.row_ptr[row + 1];
    }
    const int last_row = min(T.n_a, (rb + 1) * kWarpsPerBlock) - 1;
    const int blim = T.lower ? min(T.n_b, last_row + 1) : T.n_b;
    const int t0 = sg * TC;
    if (t0 >= blim) return;
    const int tn = min(TC, blim - t0);
    stage_cols<W>(tile, T.b, t0, tn);
    __syncthreads();
    // records for the first `cnt` queued columns
    auto drain = [&](int cnt) {
        if (lane < cnt) {
            const int cl = q[lane];
            uint64_t b[2 * W];
            tile_det<W>(tile, cl, b);
            const int deg = degree_of<W, MODE>(a, b);
            const int64_t at = pos + lane;
            if (at < end) {
                hb_pair r;
                make_record<W, MODE>(a, b, deg, T.cont_spin, row, t0 + cl, r);
                T.out[at] = r;
            }
        }
        pos += cnt;
    };
    const int cend = active ? min(tn, limit - t0) : 0;
    int qn = 0;
    for (int c0 = 0; c0 < cend; c0 += 32) {
        const int cl = c0 + lane;
        bool ok = false;
        if (cl < cend) {
            uint64_t b[2 * W];
            tile_det<W>(tile, cl, b);
            ok = degree_of<W, MODE>(a, b) <= T.max_degree;
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (ok) q[qn + __popc(m & ((1u << lane) - 1u))] = cl;
        qn += __popc(m);
        __syncwarp();
        if (qn >= 32) {
            drain(32);
            __syncwarp();
            const int rest = qn - 32;
            const int mv = lane < rest ? q[32 + lane] : 0;
            __syncwarp();
            if (lane < rest) q[lane] = mv;
            qn = rest;
            __syncwarp();
        }
    }
    if (qn > 0) drain(qn);
}

// Inclusive scan of x[1..n] in place (x[0] = 0 is set), single block.
__global__ void __launch_bounds__(1024) scan_kernel(int64_t *x, int n) {
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) { carry = 0; x[0] = 0; }
    __syncthreads();
    int64_t *y = x + 1;
    for (int base = 0; base < n; base += 1024 * 4) {
        int64_t v[4];
        const int i0 = base + tid * 4;
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (i0 + k < n) ? y[i0 + k] : 0;
        v[1] += v[0]; v[2] += v[1]; v[3] += v[2];
        int64_t t = v[3];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int64_t u = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += u;
        }
        if (lane == 31) warp_sums[warp] = t;
        __syncthreads();
        if (warp == 0) {
            int64_t s = warp_sums[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                int64_t u = __shfl_up_sync(0xffffffffu, s, off);
                if (lane >= off) s += u;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int64_t prefix = carry + (warp > 0 ? warp_sums[warp - 1] : 0) + (t - v[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i0 + k < n) y[i0 + k] = v[k] + prefix;
        __syncthreads();
        if (tid == 0) carry += warp_sums[31];
        __syncthreads();
    }
}

template <int MODE>
void count_dispatch(const uint64_t *a, int n_a, const uint64_t *b, int n_b, int W, int max_degree,
                    int lower, int64_t *counts, cudaStream_t s) {
    const dim3 grid((n_a + kWarpsPerBlock - 1) / kWarpsPerBlock), block(32 * kWarpsPerBlock);
    switch (W) {
        case 1: k1_count_kernel<1, MODE><<<grid, block, 0, s>>>(a, n_a, b, n_b, max_degree, lower, counts); break;
        case 2: k1_count_kernel<2, MODE><<<grid, block, 0, s>>>(a, n_a, b, n_b, max_degree, lower, counts); break;
        case 3: k1_count_kernel<3, MODE><<<grid, block, 0, s>>>(a, n_a, b, n_b, max_degree, lower, counts); break;
        default: k1_count_kernel<4, MODE><<<grid, block, 0, s>>>(a, n_a, b, n_b, max_degree, lower, counts); break;
    }
}

template <int MODE>
void fill_dispatch(const uint64_t *a, int n_a, const uint64_t *b, int n_b, int W, int cont_spin,
                   int max_degree, int lower, const int64_t *row_ptr, hb_pair *out, cudaStream_t s) {
    const dim3 grid((n_a + kWarpsPerBlock - 1) / kWarpsPerBlock), block(32 * kWarpsPerBlock);
    switch (W) {
        case 1: k1_fill_kernel<1, MODE><<<grid, block, 0, s>>>(a, n_a, b, n_b, cont_spin, max_degree, lower, row_ptr, out); break;
        case 2: k1_fill_kernel<2, MODE><<<grid, block, 0, s>>>(a, n_a, b, n_b, cont_spin, max_degree, lower, row_ptr, out); break;
        case 3: k1_fill_kernel<3, MODE><<<grid, block, 0, s>>>(a, n_a, b, n_b, cont_spin, max_degree, lower, row_ptr, out); break;
        default: k1_fill_kernel<4, MODE><<<grid, block, 0, s>>>(a, n_a, b, n_b, cont_spin, max_degree, lower, row_ptr, out); break;
    }
}

}  // namespace

void k1_count(const uint64_t *a, int n_a, const uint64_t *b, int n_b, int W, int mode, int max_degree,
              int lower, int64_t *counts_plus1, cudaStream_t s) {
    if (n_a <= 0) return;
    if (mode == 0) count_dispatch<0>(a, n_a, b, n_b, W, max_degree, lower, counts_plus1, s);
    else count_dispatch<1>(a, n_a, b, n_b, W, max_degree, lower, counts_plus1, s);
}

void k1_fill_pairs(const uint64_t *a, int n_a, const uint64_t *b, int n_b, int W, int mode, int cont_spin,
                   int max_degree, int lower, const int64_t *row_ptr, hb_pair *out, cudaStream_t s) {
    if (n_a <= 0) return;
    if (mode == 0) fill_dispatch<0>(a, n_a, b, n_b, W, cont_spin, max_degree, lower, row_ptr, out, s);
    else fill_dispatch<1>(a, n_a, b, n_b, W, cont_spin, max_degree, lower, row_ptr, out, s);
}

int seg_count(int n_b) { return n_b > 0 ? (n_b + kSeg - 1) / kSeg : 1; }

void k1_seg_offsets(const uint64_t *a, int n_a, const uint64_t *b, int n_b, int W, int mode, int max_degree,
                    int lower, int32_t *seg_off, cudaStream_t s) {
    if (n_a <= 0) return;
    const int nseg = seg_count(n_b);
    const unsigned grid = (unsigned)(((int64_t)n_a * nseg + kWarpsPerBlock - 1) / kWarpsPerBlock);
    const dim3 block(32 * kWarpsPerBlock);
#define HB_SEG(WW, MM) k1_seg_count_kernel<WW, MM><<<grid, block, 0, s>>>(a, n_a, b, n_b, max_degree, lower, nseg, seg_off)
    if (mode == 0) {
        switch (W) { case 1: HB_SEG(1, 0); break; case 2: HB_SEG(2, 0); break; case 3: HB_SEG(3, 0); break; default: HB_SEG(4, 0); break; }
    } else {
        switch (W) { case 1: HB_SEG(1, 1); break; case 2: HB_SEG(2, 1); break; case 3: HB_SEG(3, 1); break; default: HB_SEG(4, 1); break; }
    }
#undef HB_SEG
    seg_scan_kernel<<<(n_a + 255) / 256, 256, 0, s>>>(seg_off, n_a, nseg);
}

int64_t blocks_seg_rows8(int64_t rows, int n_b) { return ((rows + 7) / 8) * seg_count(n_b); }

void exclusive_scan_inplace(int64_t *x, int n, cudaStream_t s) {
    scan_kernel<<<1, 1024, 0, s>>>(x, n);
}

int g_classify(const Grouped<ClsTask> &g, int W, int mode, cudaStream_t s) {
    if (g.blocks <= 0) return 0;
    const dim3 grid((unsigned)g.blocks), block(32 * kWarpsPerBlock);
#define HB_K1G(WW) (mode == 0 ? k1_fill_grouped<WW, 0><<<grid, block, 0, s>>>(g.tasks, g.blk, g.n) \
                              : k1_fill_grouped<WW, 1><<<grid, block, 0, s>>>(g.tasks, g.blk, g.n))
    switch (W) {
        case 1: HB_K1G(1); break;
        case 2: HB_K1G(2); break;
        case 3: HB_K1G(3); break;
        default: HB_K1G(4); break;
    }
#undef HB_K1G
    return 1;
}

}  // namespace hb
