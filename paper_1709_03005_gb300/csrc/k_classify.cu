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

// The same over many (a, b) tasks in one launch.
template <int W, int MODE>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
k1_fill_grouped(const ClsTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const ClsTask &T = tasks[ti];
    const int row = (int)(blockIdx.x - blk[ti]) * kWarpsPerBlock + (threadIdx.x >> 5);
    if (row >= T.n_a) return;
    fill_row<W, MODE>(T.a, T.b, T.n_b, T.cont_spin, T.max_degree, T.lower, T.row_ptr, T.out, row,
                      threadIdx.x & 31);
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
