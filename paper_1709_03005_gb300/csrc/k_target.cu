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
// point atomics anywhere).
#include "hb_internal.cuh"

namespace hb {

namespace {

// ---------------------------------------------------------------- sandwich
// Wout[m][n'] = sum over records k of row m of v_k * Cp[col_k][n'].  One warp
// per row: lane l takes records l, l+32, ... (fixed order), 16 columns at a
// time, then a butterfly reduction over the lanes (fixed order as well).
__global__ void sandwich_kernel(const hb_pair *__restrict__ pairs, const int64_t *__restrict__ row_ptr,
                                const double *__restrict__ val, int n_rows, const double *__restrict__ Cp, int nsp,
                                double *__restrict__ Wout) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n_rows) return;
    const int64_t b = row_ptr[row], e = row_ptr[row + 1];
    for (int n0 = 0; n0 < nsp; n0 += 16) {
        double acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = 0.0;
        for (int64_t k = b + lane; k < e; k += 32) {
            const int col = pairs[k].col;
            const double v = val[k];
            const double *crow = Cp + (int64_t)col * nsp + n0;
#pragma unroll
            for (int c = 0; c < 16; ++c)
                if (n0 + c < nsp) acc[c] = fma(v, __ldg(crow + c), acc[c]);
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) {
#pragma unroll
            for (int off = 16; off; off >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
        }
        if (lane < 16 && n0 + lane < nsp) {
            double mine = 0.0;
#pragma unroll
            for (int c = 0; c < 16; ++c)
                if (c == lane) mine = acc[c];
            Wout[(int64_t)row * nsp + n0 + lane] = mine;
        }
    }
}

// partial[c][n][n'] = sum_{m in chunk c} C[m][n] * Wm[m][n']; rows staged in
// batches of 32, each thread keeps 4 outputs, grid.y covers the outputs.
constexpr int kRowsPerChunk = 256;
// rows (or items) staged per batch so that the staging buffer stays <= 48 KB
__host__ __device__ inline int stage_batch(int ns, int nsp) {
    const int b = 6144 / (ns + nsp);
    return b < 1 ? 1 : (b > 32 ? 32 : b);
}
__global__ void tn_partial_kernel(const double *__restrict__ C, const double *__restrict__ Wm, int n_rows,
                                  int ns, int nsp, double *__restrict__ partial) {
    extern __shared__ double sh[];
    const int kRowBatch = stage_batch(ns, nsp);
    double *cs = sh;                      // [kRowBatch][ns]
    double *ws = sh + kRowBatch * ns;     // [kRowBatch][nsp]
    const int c = blockIdx.x;
    const int m0 = c * kRowsPerChunk;
    const int rows = min(kRowsPerChunk, n_rows - m0);
    const int nout = ns * nsp;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r0 = 0; r0 < rows; r0 += kRowBatch) {
        const int nr = min(kRowBatch, rows - r0);
        __syncthreads();
        for (int i = threadIdx.x; i < nr * ns; i += blockDim.x) cs[i] = C[(int64_t)(m0 + r0) * ns + i];
        for (int i = threadIdx.x; i < nr * nsp; i += blockDim.x) ws[i] = Wm[(int64_t)(m0 + r0) * nsp + i];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = blockIdx.y * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
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
        const int t = blockIdx.y * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
        if (t < nout) partial[(int64_t)c * nout + t] = acc[u];
    }
}

__global__ void reduce_partials_kernel(const double *__restrict__ partial, int n_chunks, int n_out,
                                       double *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_out) return;
    double acc = 0.0;
    for (int c = 0; c < n_chunks; ++c) acc += partial[(int64_t)c * n_out + t];
    out[t] = acc;
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
        cnt += d == 0 ? n_elec : (d == 1 ? 1 : 0);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    if (lane == 0) counts_plus1[row + 1] = cnt;
}

// Items in record order; a deg-0 record emits its occupied spin orbitals in
// canonical order.  key = spin * n_to^2 + r * n_to + q.
__global__ void item_fill_kernel(const hb_pair *__restrict__ pairs, const int64_t *__restrict__ row_ptr,
                                 int n_rows, const uint64_t *__restrict__ bra_dets, int W, int n_to, int n_elec,
                                 const int64_t *__restrict__ item_ptr, GammaItem *__restrict__ items) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n_rows) return;
    const int64_t b = row_ptr[row], e = row_ptr[row + 1];
    int64_t pos = item_ptr[row];
    const int sb = 64 * W;
    for (int64_t k0 = b; k0 < e; k0 += 32) {
        const int64_t k = k0 + lane;
        int cnt = 0;
        hb_pair r;
        if (k < e) {
            r = pairs[k];
            cnt = r.degree == 0 ? n_elec : (r.degree == 1 ? 1 : 0);
        }
        int incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += u;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int64_t at = pos + (incl - cnt);
        if (cnt) {
            if (r.degree == 1) {
                const int s = r.part[0] / sb, p = r.part[0] % sb, q = r.hole[0] % sb;
                GammaItem it;
                it.key = s * n_to * n_to + p * n_to + q;
                it.m = r.row; it.mp = r.col; it.phase = r.phase;
                items[at] = it;
            } else {
                const uint64_t *d = bra_dets + (int64_t)r.row * 2 * W;
                for (int w = 0; w < 2 * W; ++w) {
                    uint64_t x = d[w];
                    while (x) {
                        const int bit = 64 * w + __ffsll((long long)x) - 1;
                        x &= x - 1;
                        const int s = bit / sb, p = bit % sb;
                        GammaItem it;
                        it.key = s * n_to * n_to + p * n_to + p;
                        it.m = r.row; it.mp = r.col; it.phase = 1;
                        items[at++] = it;
                    }
                }
            }
        }
        pos += total;
    }
}

// ------------------------------------------------- stable counting sort by key
constexpr int kSortChunk = 4096;

__global__ void sort_hist_kernel(const GammaItem *__restrict__ items, int64_t n_items, int n_chunks,
                                 unsigned long long *__restrict__ hist_plus1) {
    const int64_t base = (int64_t)blockIdx.x * kSortChunk;
    for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x) {
        const int64_t k = base + i;
        if (k < n_items) atomicAdd(hist_plus1 + 1 + (int64_t)items[k].key * n_chunks + blockIdx.x, 1ull);
    }
}

// One warp per chunk walks its items in order, so equal keys keep their order.
// cursors: a copy of the exclusive offsets [key][chunk], advanced in place.
__global__ void sort_scatter_kernel(const GammaItem *__restrict__ items, int64_t n_items, int n_chunks,
                                    int64_t *__restrict__ cursors, int32_t *__restrict__ order) {
    const int lane = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * kSortChunk;
    for (int i0 = 0; i0 < kSortChunk; i0 += 32) {
        const int64_t k = base + i0 + lane;
        const bool valid = k < n_items;
        const int key = valid ? items[k].key : -1 - lane;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const int leader = __ffs(peers) - 1;
        int64_t *cur = valid ? cursors + (int64_t)key * n_chunks + blockIdx.x : nullptr;
        int64_t at = 0;
        if (valid) at = *cur + rank;
        __syncwarp();
        if (valid && lane == leader) *cur += __popc(peers);
        __syncwarp();
        if (valid) order[at] = (int32_t)k;
    }
}

// gamma[key][n][n'] = sum over the key's items of phase * C[m][n] * Cp[m'][n']
__global__ void gamma_kernel(const GammaItem *__restrict__ items, const int32_t *__restrict__ order,
                             const int64_t *__restrict__ offsets, int n_chunks, int64_t n_items,
                             const double *__restrict__ C, int ns, const double *__restrict__ Cp, int nsp,
                             double *__restrict__ gamma) {
    extern __shared__ double sm[];
    const int kItemBatch = stage_batch(ns, nsp);
    double *ca = sm;                          // [kItemBatch][ns]
    double *cb = sm + kItemBatch * ns;        // [kItemBatch][nsp]
    const int key = blockIdx.x;
    const int64_t b = offsets[(int64_t)key * n_chunks];
    const int64_t e = offsets[(int64_t)(key + 1) * n_chunks];
    const int nout = ns * nsp;
    // each thread keeps up to 4 outputs in registers
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i0 = b; i0 < e; i0 += kItemBatch) {
        const int cnt = (int)(e - i0 < kItemBatch ? e - i0 : kItemBatch);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt * ns; t += blockDim.x) {
            const int i = t / ns, a = t % ns;
            const GammaItem it = items[order[i0 + i]];
            ca[i * ns + a] = it.phase * C[(int64_t)it.m * ns + a];
        }
        for (int t = threadIdx.x; t < cnt * nsp; t += blockDim.x) {
            const int i = t / nsp, a = t % nsp;
            const GammaItem it = items[order[i0 + i]];
            cb[i * nsp + a] = Cp[(int64_t)it.mp * nsp + a];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = blockIdx.y * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
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
        const int t = blockIdx.y * 4 * blockDim.x + u * blockDim.x + threadIdx.x;
        if (t < nout) gamma[(int64_t)key * nout + t] = acc[u];
    }
}

// ------------------------------------------------------ coefficient rows
// A[t][k] for the state pairs t = (n, n'):
//   k <  Pt            : Gamma^(r>=s) = sum_spin gamma(r,s) + gamma(s,r) (r != s)
//   Pt <= k < Pt+n_to^2: -gamma^{cont spin}(p, q)
//   k == Pt+n_to^2     : S            (multiplies h_jj')
//   k == Pt+n_to^2+1   : E + e_core S (multiplies delta_jj')
//   k >= K             : 0
__global__ void assemble_kernel(const double *__restrict__ gamma, const double *__restrict__ S,
                                const double *__restrict__ E, const int32_t *__restrict__ nn, int n_nn, int ns,
                                int nsp, int n_to, int cont_spin, double e_core, int Kpad,
                                double *__restrict__ A) {
    const int t = blockIdx.x;
    if (t >= n_nn) return;
    const int n = nn[2 * t], np = nn[2 * t + 1];
    const int nout = ns * nsp, sidx = n * nsp + np;
    const int Pt = n_to * (n_to + 1) / 2, nt2 = n_to * n_to;
    for (int k = threadIdx.x; k < Kpad; k += blockDim.x) {
        double v = 0.0;
        if (k < Pt) {
            // unpack k = r(r+1)/2 + s
            int r = (int)((sqrt(8.0 * k + 1.0) - 1.0) * 0.5);
            while ((r + 1) * (r + 2) / 2 <= k) ++r;
            while (r * (r + 1) / 2 > k) --r;
            const int s = k - r * (r + 1) / 2;
            for (int sp = 0; sp < 2; ++sp) {
                v += gamma[((int64_t)sp * nt2 + r * n_to + s) * nout + sidx];
                if (r != s) v += gamma[((int64_t)sp * nt2 + s * n_to + r) * nout + sidx];
            }
        } else if (k < Pt + nt2) {
            const int pq = k - Pt;
            v = -gamma[((int64_t)cont_spin * nt2 + pq) * nout + sidx];
        } else if (k == Pt + nt2) {
            v = S[sidx];
        } else if (k == Pt + nt2 + 1) {
            v = E[sidx] + e_core * S[sidx];
        }
        A[(int64_t)t * Kpad + k] = v;
    }
}

}  // namespace

void sandwich_rows(const hb_pair *pairs, const int64_t *row_ptr, const double *val, int n_rows, const double *Cp,
                   int nsp, double *Wout, cudaStream_t s) {
    if (n_rows <= 0) return;
    sandwich_kernel<<<(n_rows + 7) / 8, 256, 0, s>>>(pairs, row_ptr, val, n_rows, Cp, nsp, Wout);
}

int tn_chunks(int n_rows) { return (n_rows + kRowsPerChunk - 1) / kRowsPerChunk; }

void gemm_tn_reduce(const double *C, const double *Wm, int n_rows, int ns, int nsp, double *partials,
                    double *out, cudaStream_t s) {
    const int nc = tn_chunks(n_rows);
    if (nc > 0) {
        const size_t sh = sizeof(double) * stage_batch(ns, nsp) * (ns + nsp);
        const dim3 grid(nc, (ns * nsp + 1023) / 1024);
        tn_partial_kernel<<<grid, 256, sh, s>>>(C, Wm, n_rows, ns, nsp, partials);
    }
    const int n_out = ns * nsp;
    reduce_partials_kernel<<<(n_out + 255) / 256, 256, 0, s>>>(partials, nc, n_out, out);
}

void gamma_item_counts(const hb_pair *pairs, const int64_t *row_ptr, int n_rows, int n_elec,
                       int64_t *counts_plus1, cudaStream_t s) {
    if (n_rows <= 0) return;
    item_count_kernel<<<(n_rows + 7) / 8, 256, 0, s>>>(pairs, row_ptr, n_rows, n_elec, counts_plus1);
}

void gamma_item_fill(const hb_pair *pairs, const int64_t *row_ptr, int n_rows, const uint64_t *bra_dets, int W,
                     int n_to, int n_elec, const int64_t *item_ptr, GammaItem *items, cudaStream_t s) {
    if (n_rows <= 0) return;
    item_fill_kernel<<<(n_rows + 7) / 8, 256, 0, s>>>(pairs, row_ptr, n_rows, bra_dets, W, n_to, n_elec, item_ptr,
                                                      items);
}

int sort_chunks(int64_t n_items) { return (int)((n_items + kSortChunk - 1) / kSortChunk); }

void gamma_sort(const GammaItem *items, int64_t n_items, int n_keys, int64_t *offsets_plus1, int64_t *cursors,
                int32_t *order, cudaStream_t s) {
    const int nc = sort_chunks(n_items);
    const int64_t n_off = (int64_t)n_keys * nc;
    // zero the histogram (also covers the n_items == 0 case)
    cudaMemsetAsync(offsets_plus1, 0, sizeof(int64_t) * (n_off + 1), s);
    if (nc > 0) {
        sort_hist_kernel<<<nc, 256, 0, s>>>(items, n_items, nc, (unsigned long long *)offsets_plus1);
        exclusive_scan_inplace(offsets_plus1, (int)n_off, s);
        cudaMemcpyAsync(cursors, offsets_plus1, sizeof(int64_t) * n_off, cudaMemcpyDeviceToDevice, s);
        sort_scatter_kernel<<<nc, 32, 0, s>>>(items, n_items, nc, cursors, order);
    }
}

void gamma_bins(const GammaItem *items, const int32_t *order, const int64_t *offsets, int n_keys, int64_t n_items,
                const double *C, int ns, const double *Cp, int nsp, double *gamma, cudaStream_t s) {
    const int nc = sort_chunks(n_items);
    if (nc == 0) {
        cudaMemsetAsync(gamma, 0, sizeof(double) * (size_t)n_keys * ns * nsp, s);
        return;
    }
    // each thread holds 4 outputs, grid.y covers ns * nsp in steps of 1024
    const size_t sh = sizeof(double) * stage_batch(ns, nsp) * (ns + nsp);
    const dim3 grid(n_keys, (ns * nsp + 1023) / 1024);
    gamma_kernel<<<grid, 256, sh, s>>>(items, order, offsets, nc, n_items, C, ns, Cp, nsp, gamma);
}

void assemble_coefficients(const double *gamma, const double *S, const double *E, const int32_t *nn, int n_nn,
                           int ns, int nsp, int n_to, int cont_spin, double e_core, int Kpad, double *A,
                           cudaStream_t s) {
    if (n_nn <= 0) return;
    assemble_kernel<<<n_nn, 256, 0, s>>>(gamma, S, E, nn, n_nn, ns, nsp, n_to, cont_spin, e_core, Kpad, A);
}

}  // namespace hb
