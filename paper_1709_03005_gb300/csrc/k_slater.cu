// K5: numeric Slater-Condon elements between target-orbital determinants
// (classes 2 and 8, the L2 x L2 block, Section 2.2; and the target Hamiltonian
// H^N used by the contraction of classes 1, 3, 5, 6, 7).
//
// diagonal : sum_i h_ii + sum_{i<k} [(ii|kk) - delta_spin (ik|ki)]
// single   : phase * [h_ph + sum_{k common} ((ph|kk) - delta_spin (pk|kh))]
// double   : phase * [(p1 h1|p2 h2) - (p1 h2|p2 h1)], with spin deltas
// (the standard rules for an orthonormal spin-orbital basis; the paper
// evaluates them symbolically, Eq. 6).  (pp|qq) and (pq|qp) come from a small
// n_to x n_to table that stays in L1/L2; other (tt|tt) integrals are gathered.
#include "hb_df.cuh"
#include "hb_tasks.cuh"

namespace hb {

namespace {

__device__ __forceinline__ double eri4(const Ints &I, int p, int q, int r, int s) {
    return __ldg(I.tttt + pair_idx(p, q) * I.Pt + pair_idx(r, s));
}

__device__ __forceinline__ int64_t eri_idx(const Ints &I, int p, int q, int r, int s) {
    return pair_idx(p, q) * I.Pt + pair_idx(r, s);
}

// Sums below run through an accumulator: AccD (FP64) or AccF (double-float
// over the float-pair tables), the same terms in the same order.
template <int W, class Acc>
__device__ Acc diag_value(const Ints &I, const uint64_t (&d)[2 * W]) {
    const int n = I.n_to, no = I.n_orb;
    const int64_t nn = (int64_t)n * n;
    Acc e;
    // one-electron and same-spin / opposite-spin pair sums
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint64_t x = d[s * W + w];
            while (x) {
                const int p = 64 * w + __ffsll((long long)x) - 1;
                x &= x - 1;
                e.add(I.h, I.h_df, (int64_t)p * no + p);
                // pairs (p, q) with q after p in canonical order
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    if (s2 < s) continue;
#pragma unroll
                    for (int w2 = 0; w2 < W; ++w2) {
                        uint64_t y = d[s2 * W + w2];
                        if (s2 == s) {
                            if (w2 < w) continue;
                            if (w2 == w) y &= x;  // bits above p in the same word (x already cleared p)
                        }
                        while (y) {
                            const int q = 64 * w2 + __ffsll((long long)y) - 1;
                            y &= y - 1;
                            e.add(I.jk, I.jk_df, (int64_t)p * n + q);
                            if (s2 == s) e.sub(I.jk, I.jk_df, nn + (int64_t)p * n + q);
                        }
                    }
                }
            }
        }
    }
    return e;
}

template <int W, class Acc>
__device__ Acc single_value(const Ints &I, const uint64_t (&bra)[2 * W], const uint64_t (&ket)[2 * W], int hpos,
                            int ppos) {
    const int sb = 64 * W;
    const int hs = hpos / sb, h = hpos % sb, p = ppos % sb;
    Acc v;
    v.add(I.h, I.h_df, (int64_t)p * I.n_orb + h);
    const int64_t ph = pair_idx(p, h) * I.Pt;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint64_t x = bra[s * W + w] & ket[s * W + w];
            while (x) {
                const int k = 64 * w + __ffsll((long long)x) - 1;
                x &= x - 1;
                v.add(I.tttt, I.tttt_df, ph + pair_idx(k, k));
                if (s == hs) v.sub(I.tttt, I.tttt_df, eri_idx(I, p, k, k, h));
            }
        }
    }
    return v;
}

template <class Acc>
__device__ __forceinline__ Acc double_value(const Ints &I, int W, int h1, int h2, int p1, int p2) {
    const int sb = 64 * W;
    Acc v;
    if (p1 / sb == h1 / sb && p2 / sb == h2 / sb) v.add(I.tttt, I.tttt_df, eri_idx(I, p1 % sb, h1 % sb, p2 % sb, h2 % sb));
    if (p1 / sb == h2 / sb && p2 / sb == h1 / sb) v.sub(I.tttt, I.tttt_df, eri_idx(I, p1 % sb, h2 % sb, p2 % sb, h1 % sb));
    return v;
}

template <int W>
__device__ __forceinline__ void load_det(const uint64_t *p, uint64_t (&x)[2 * W]) {
#pragma unroll
    for (int i = 0; i < 2 * W; ++i) x[i] = __ldg(p + i);
}

template <int W>
__device__ __forceinline__ int diff_bits(const uint64_t (&x)[2 * W], const uint64_t (&y)[2 * W], int (&pos)[2]) {
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

// Full element <bra|H|ket> (same electron count), classification inline.
template <int W, class Acc>
__device__ Acc element(const Ints &I, const uint64_t (&a)[2 * W], const uint64_t (&b)[2 * W], int deg) {
    if (deg == 0) return diag_value<W, Acc>(I, a);
    int h[2], p[2];
    diff_bits<W>(b, a, h);
    diff_bits<W>(a, b, p);
    if (deg == 1) {
        const int e = prefix_count(b, 2 * W, h[0]) + prefix_count(b, 2 * W, p[0]) - (h[0] < p[0]);
        Acc v = single_value<W, Acc>(I, a, b, h[0], p[0]);
        if (e & 1) v.neg();
        return v;
    }
    const int e = prefix_count(b, 2 * W, h[0]) + prefix_count(b, 2 * W, h[1]) - 1 + prefix_count(b, 2 * W, p[1]) -
                  (h[0] < p[1]) - (h[1] < p[1]) + prefix_count(b, 2 * W, p[0]) - (h[0] < p[0]) - (h[1] < p[0]);
    Acc v = double_value<Acc>(I, W, h[0], h[1], p[0], p[1]);
    if (e & 1) v.neg();
    return v;
}

__device__ __forceinline__ void store_value(const AccD &v, double *out, int64_t k) { out[k] = v.v; }
__device__ __forceinline__ void store_value(const AccF &v, double *out, int64_t k) {
    reinterpret_cast<float2 *>(out)[k] = make_float2(v.h, v.l);
}

constexpr int kWarps = 8;

// Block = 8 rows (one warp each) x one segment of kSegCols columns, staged
// through shared memory word-major (conflict-free lane reads); the segment's
// output offset within each row comes from the staging-time segment counts.
// Matches are queued per warp in column order and evaluated 32 at a time,
// one per lane.
template <int W, class Acc>
__global__ void __launch_bounds__(32 * kWarps)
l2_csr_kernel(const L2Task *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    constexpr int TC = kSegCols;
    __shared__ uint64_t tile[TC * 2 * W];
    __shared__ int queue[kWarps][64];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const L2Task &T = tasks[ti];
    const Ints I = T.I;
    const uint64_t *__restrict__ D = T.dets;
    const int n = T.n;
    const int lb = (int)(blockIdx.x - blk[ti]);
    const int rb = lb / T.nseg, sg = lb % T.nseg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row = rb * kWarps + warp;
    // a block whose rows are all outside this build's rows has nothing to do
    if (rb * kWarps >= T.row_hi || (rb + 1) * kWarps <= T.row_lo) return;
    const bool active = row < n && row >= T.row_lo && row < T.row_hi;
    int *q = queue[warp];
    uint64_t a[2 * W];
    int64_t pos = 0, end = 0;
    if (active) {
        load_det<W>(D + (int64_t)row * 2 * W, a);
        pos = T.row_ptr[row] + T.seg_off[(int64_t)row * T.nseg + sg];
        end = T.row_ptr[row + 1];
        if (lane == 0 && sg == 0) {
            T.row_ptr_out[row] = T.row_ptr[row];
            if (row == n - 1) T.row_ptr_out[n] = end;
        }
    }
    const int t0 = sg * TC;
    if (t0 >= n) return;
    const int tn = min(TC, n - t0);
    // upper triangle only: a segment below the diagonal of every row of the block has nothing to do
    if (T.low_ptr && t0 + tn <= rb * kWarps) return;
    for (int i = threadIdx.x; i < tn * 2 * W; i += blockDim.x) {
        const int c = i / (2 * W), w = i % (2 * W);
        tile[w * TC + c] = __ldg(D + (int64_t)t0 * 2 * W + i);
    }
    __syncthreads();
    if (!active) return;
    int cmin = 0;             // first column of the segment evaluated in this row
    if (T.low_ptr) {
        if (t0 + tn <= row) return;
        if (t0 <= row) {
            // the diagonal's segment: the entries of this row from the diagonal on
            cmin = row - t0;
            pos = T.row_ptr[row] + (T.low_ptr[row + 1] - T.low_ptr[row]);
        }
    }
    auto drain = [&](int cnt) {
        if (lane < cnt) {
            const int cl = q[lane];
            uint64_t b[2 * W];
            int x = 0;
#pragma unroll
            for (int i = 0; i < 2 * W; ++i) {
                b[i] = tile[i * TC + cl];
                x += __popcll(a[i] ^ b[i]);
            }
            const int deg = x >> 1;
            const int64_t at = pos + lane;
            if (at < end) {
                Acc v = element<W, Acc>(I, a, b, deg);
                if (deg == 0) v.add_const(T.e_core);
                T.col[at] = t0 + cl;
                T.val[at] = v.value();
            }
        }
        pos += cnt;
    };
    int qn = 0;
    for (int c0 = 0; c0 < tn; c0 += 32) {
        const int cl = c0 + lane;
        bool ok = false;
        if (cl < tn && cl >= cmin) {
            int x = 0;
#pragma unroll
            for (int i = 0; i < 2 * W; ++i) x += __popcll(a[i] ^ tile[i * TC + cl]);
            ok = (x >> 1) <= 2;
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

// The L2 x L2 block is symmetric (the excitation test and the Slater-Condon
// value do not depend on the order of the pair), so a build evaluates the
// entries with col >= row and copies each entry below the diagonal from its
// mirror.  The positions depend only on the determinants; the kernels after
// this one find them once per context.
__global__ void l2_mirror_kernel(const L2MTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const L2MTask &T = tasks[ti];
    const int64_t i = (int64_t)(blockIdx.x - blk[ti]) * kL2MirrorThreads + threadIdx.x;
    if (i >= T.n) return;
    const int c = T.mcol[i];
    if (c < T.src_lo || c >= T.src_hi) return;
    const int64_t d = T.dst[i];
    T.col[d] = c;
    T.val[d] = T.val[T.src[i]];
}

// One warp per row: the columns of its entries in ascending order.
template <int W>
__global__ void l2_struct_kernel(const uint64_t *__restrict__ D, int n, const int64_t *__restrict__ row_ptr,
                                 int32_t *__restrict__ col) {
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    uint64_t a[2 * W];
    load_det<W>(D + row * 2 * W, a);
    int64_t pos = row_ptr[row];
    const int64_t end = row_ptr[row + 1];
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int c = c0 + lane;
        bool ok = false;
        if (c < n) {
            int x = 0;
#pragma unroll
            for (int i = 0; i < 2 * W; ++i) x += __popcll(a[i] ^ __ldg(D + (int64_t)c * 2 * W + i));
            ok = (x >> 1) <= 2;
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        const int64_t at = pos + __popc(m & ((1u << lane) - 1u));
        if (ok && at < end) col[at] = c;
        pos += __popc(m);
    }
}

// First position in [b, e) whose column is >= c (columns ascending).
__device__ __forceinline__ int64_t lower_bound_col(const int32_t *__restrict__ col, int64_t b, int64_t e, int c) {
    while (b < e) {
        const int64_t m = b + ((e - b) >> 1);
        if (col[m] < c) b = m + 1;
        else e = m;
    }
    return b;
}

__global__ void l2_lower_counts_kernel(const int32_t *__restrict__ col, const int64_t *__restrict__ row_ptr, int n,
                                       int64_t *__restrict__ low_ptr) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    low_ptr[r + 1] = lower_bound_col(col, row_ptr[r], row_ptr[r + 1], r) - row_ptr[r];
}

// One thread per entry below the diagonal (nl of them, in row order): its row
// by binary search over the prefix, then its mirror by binary search in the
// row of its column.
__global__ void l2_mirror_fill_kernel(const int32_t *__restrict__ col, const int64_t *__restrict__ row_ptr, int n,
                                      const int64_t *__restrict__ low_ptr, int64_t nl, int64_t *__restrict__ dst,
                                      int64_t *__restrict__ src, int32_t *__restrict__ mcol, int *missing) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0 && low_ptr[n] != nl) atomicExch(missing, 1);
    if (q >= nl) return;
    if (q >= low_ptr[n]) {
        atomicExch(missing, 1);
        return;
    }
    int lo = 0, hi = n;      // the last row r with low_ptr[r] <= q
    while (hi - lo > 1) {
        const int mid = lo + ((hi - lo) >> 1);
        if (low_ptr[mid] <= q) lo = mid;
        else hi = mid;
    }
    const int r = lo;
    const int64_t at = row_ptr[r] + (q - low_ptr[r]);
    const int c = col[at];
    int64_t m = at;
    if (c < 0 || c >= r) {
        atomicExch(missing, 1);          // not below the diagonal: the lists stay unused
    } else {
        const int64_t e = row_ptr[c + 1];
        m = lower_bound_col(col, row_ptr[c], e, r);
        if (m >= e || col[m] != r) {
            atomicExch(missing, 1);
            m = at;
        }
    }
    dst[q] = at;
    src[q] = m;
    mcol[q] = c;
}

// <A[row]|H|B[col]> for classified pairs (mode 0 records).  FP64: val as
// doubles; double-float: val as (hi, lo) float pairs in the same 8 bytes.
template <int W, class Acc>
__global__ void pair_values_kernel(const PVTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const PVTask &T = tasks[ti];
    const int64_t k = (blockIdx.x - blk[ti]) * (int64_t)blockDim.x + threadIdx.x;
    if (k >= T.n_pairs) return;
    const Ints I = T.I;
    const hb_pair r = T.pairs[k];
    // within one group the diagonal records (O(N^2) sums, one per row) are
    // left to diag_values_kernel, so that no warp here waits on one
    if (r.degree == 0 && T.same) return;
    uint64_t a[2 * W], b[2 * W];
    load_det<W>(T.a + (int64_t)r.row * 2 * W, a);
    load_det<W>(T.b + (int64_t)r.col * 2 * W, b);
    Acc v;
    if (r.degree == 0) v = diag_value<W, Acc>(I, a);
    else if (r.degree == 1) v = single_value<W, Acc>(I, a, b, r.hole[0], r.part[0]);
    else v = double_value<Acc>(I, W, r.hole[0], r.hole[1], r.part[0], r.part[1]);
    if (r.degree > 0 && r.phase < 0) v.neg();
    store_value(v, T.val, k);
}

// <D_m|H^N|D_m> of a same-group task: the record (m, m) of row m, found by
// binary search over the row's ascending columns (a scan if that fails).
template <int W, class Acc>
__global__ void diag_values_kernel(const PVTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const PVTask &T = tasks[ti];
    const int m = (int)((blockIdx.x - blk[ti]) * (int64_t)blockDim.x + threadIdx.x);
    if (m >= T.n_rows) return;
    int64_t lo = T.row_ptr[m], hi = T.row_ptr[m + 1] - 1, at = -1;
    while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int c = T.pairs[mid].col;
        if (c == m) { at = mid; break; }
        if (c < m) lo = mid + 1;
        else hi = mid - 1;
    }
    if (at < 0)
        for (int64_t k = T.row_ptr[m]; k < T.row_ptr[m + 1]; ++k)
            if (T.pairs[k].col == m) { at = k; break; }
    if (at < 0 || T.pairs[at].degree != 0) return;
    uint64_t a[2 * W];
    load_det<W>(T.a + (int64_t)m * 2 * W, a);
    store_value(diag_value<W, Acc>(T.I, a), T.val, at);
}

__global__ void jk_kernel(Ints I, double *jk) {
    const int n = I.n_to;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * n) return;
    const int p = t / n, q = t % n;
    jk[t] = eri4(I, p, p, q, q);
    jk[n * n + t] = eri4(I, p, q, q, p);
}

}  // namespace

void build_jk(const Ints &I, double *jk, cudaStream_t s) {
    const int n = I.n_to * I.n_to;
    jk_kernel<<<(n + 255) / 256, 256, 0, s>>>(I, jk);
}

int64_t blocks_pair_values(int64_t n_pairs) { return (n_pairs + 255) / 256; }
int64_t blocks_diag_values(int n_rows) { return (n_rows + 255) / 256; }

int g_diag_values(const Grouped<PVTask> &g, int W, int dfloat, cudaStream_t s) {
    if (g.blocks <= 0) return 0;
    const unsigned grid = (unsigned)g.blocks;
#define HB_DV(WW) (dfloat ? diag_values_kernel<WW, AccF><<<grid, 256, 0, s>>>(g.tasks, g.blk, g.n) \
                          : diag_values_kernel<WW, AccD><<<grid, 256, 0, s>>>(g.tasks, g.blk, g.n))
    switch (W) {
        case 1: HB_DV(1); break;
        case 2: HB_DV(2); break;
        case 3: HB_DV(3); break;
        default: HB_DV(4); break;
    }
#undef HB_DV
    return 1;
}

int g_l2_csr(const Grouped<L2Task> &g, int W, int dfloat, cudaStream_t s) {
    if (g.blocks <= 0) return 0;
    const dim3 grid((unsigned)g.blocks), block(32 * kWarps);
#define HB_L2(WW) (dfloat ? l2_csr_kernel<WW, AccF><<<grid, block, 0, s>>>(g.tasks, g.blk, g.n) \
                          : l2_csr_kernel<WW, AccD><<<grid, block, 0, s>>>(g.tasks, g.blk, g.n))
    switch (W) {
        case 1: HB_L2(1); break;
        case 2: HB_L2(2); break;
        case 3: HB_L2(3); break;
        default: HB_L2(4); break;
    }
#undef HB_L2
    return 1;
}

int g_l2_mirror(const Grouped<L2MTask> &g, cudaStream_t s) {
    if (g.blocks <= 0) return 0;
    l2_mirror_kernel<<<(unsigned)g.blocks, kL2MirrorThreads, 0, s>>>(g.tasks, g.blk, g.n);
    return 1;
}

void l2_struct(const uint64_t *dets, int n, int W, const int64_t *row_ptr, int32_t *col, cudaStream_t s) {
    if (n <= 0) return;
    const unsigned grid = (unsigned)(((int64_t)n * 32 + 255) / 256);
    switch (W) {
        case 1: l2_struct_kernel<1><<<grid, 256, 0, s>>>(dets, n, row_ptr, col); break;
        case 2: l2_struct_kernel<2><<<grid, 256, 0, s>>>(dets, n, row_ptr, col); break;
        case 3: l2_struct_kernel<3><<<grid, 256, 0, s>>>(dets, n, row_ptr, col); break;
        default: l2_struct_kernel<4><<<grid, 256, 0, s>>>(dets, n, row_ptr, col); break;
    }
}

void l2_lower_counts(const int32_t *col, const int64_t *row_ptr, int n, int64_t *low_ptr, cudaStream_t s) {
    if (n <= 0) return;
    l2_lower_counts_kernel<<<(n + 255) / 256, 256, 0, s>>>(col, row_ptr, n, low_ptr);
}

void l2_mirror_fill(const int32_t *col, const int64_t *row_ptr, int n, const int64_t *low_ptr, int64_t nl,
                    int64_t *dst, int64_t *src, int32_t *mcol, int *missing, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t blocks = nl > 0 ? (nl + 255) / 256 : 1;
    l2_mirror_fill_kernel<<<(unsigned)blocks, 256, 0, s>>>(col, row_ptr, n, low_ptr, nl, dst, src, mcol, missing);
}

int g_pair_values(const Grouped<PVTask> &g, int W, int dfloat, cudaStream_t s) {
    if (g.blocks <= 0) return 0;
    const unsigned grid = (unsigned)g.blocks;
#define HB_PV(WW) (dfloat ? pair_values_kernel<WW, AccF><<<grid, 256, 0, s>>>(g.tasks, g.blk, g.n) \
                          : pair_values_kernel<WW, AccD><<<grid, 256, 0, s>>>(g.tasks, g.blk, g.n))
    switch (W) {
        case 1: HB_PV(1); break;
        case 2: HB_PV(2); break;
        case 3: HB_PV(3); break;
        default: HB_PV(4); break;
    }
#undef HB_PV
    return 1;
}

}  // namespace hb
