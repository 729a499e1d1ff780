// K3: expansion of the contracted prototype labels over the continuum orbitals
// (Eq. 7) for classes 1, 3, 5, 6, 7, double-precision path.
//
// With the contracted coefficients A[(n,n')][k] of K2 and the integral panel
// P[(j,j')][k] (one row per continuum pair, one column per label):
//   H~[(g n j), (g' n' j')] = sum_k P[(j,j')][k] * A[(n,n')][k]
// labels k: (jj'|rs) for r >= s, (jq|pj') for all (p, q), h_jj', delta_jj'.
// This file builds the panel (once, at staging) and runs the FP64 contraction
// with a scatter epilogue into the full symmetric continuum block.
#include "hb_tasks.cuh"

namespace hb {

namespace {

// The panel value of label k for the continuum pair (j, jp): (jj'|rs) for
// the target pair k < Pt, (jq|pj') for k = Pt + p n_to + q, h_jj', delta_jj'.
__device__ __forceinline__ double label_value(const double *__restrict__ ttcc, const double *__restrict__ tctc,
                                              const double *__restrict__ h, int n_to, int n_co, int k, int j, int jp) {
    const int Pt = n_to * (n_to + 1) / 2, nt2 = n_to * n_to, n_orb = n_to + n_co;
    const int64_t NTC = (int64_t)n_to * n_co, NCC = (int64_t)n_co * n_co;
    if (k < 0) return 0.0;
    if (k < Pt) return ttcc[(int64_t)k * NCC + (int64_t)j * n_co + jp];
    if (k < Pt + nt2) {
        const int pq = k - Pt, p = pq / n_to, q = pq % n_to;
        return tctc[((int64_t)q * n_co + j) * NTC + (int64_t)p * n_co + jp];
    }
    if (k == Pt + nt2) return h[(int64_t)(n_to + j) * n_orb + n_to + jp];
    if (k == Pt + nt2 + 1) return (j == jp) ? 1.0 : 0.0;
    return 0.0;
}

// P[(j*n_co + jp)][kk], tiles of 32 continuum orbitals jp x 32 columns kk for
// one j, transposed through shared memory so the writes are coalesced.
// Without orbital symmetry column kk is label kk.  With it, column kk of the
// row (j, jp) is the kk-th label of the class irrep(j) ^ irrep(jp) (the
// labels whose target pair has that symmetry; the others vanish on this row).
__global__ void panel_kernel(const double *__restrict__ ttcc, const double *__restrict__ tctc,
                             const double *__restrict__ h, int n_to, int n_co, int Kc,
                             const int32_t *__restrict__ cls_labels, const int32_t *__restrict__ co_irrep,
                             double *__restrict__ P) {
    __shared__ double tile[32][33];
    const int jp0 = blockIdx.x * 32, k0 = blockIdx.y * 32, j = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int kk = k0 + r, jp = jp0 + tx;
        double v = 0.0;
        if (jp < n_co) {
            const int k = cls_labels ? cls_labels[(co_irrep[j] ^ co_irrep[jp]) * Kc + kk] : kk;
            v = label_value(ttcc, tctc, h, n_to, n_co, k, j, jp);
        }
        tile[r][tx] = v;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int jp = jp0 + r, kk = k0 + tx;
        if (jp < n_co && kk < Kc) P[((int64_t)j * n_co + jp) * Kc + kk] = tile[tx][r];
    }
}

// With orbital symmetry: flag any nonzero panel value of a label outside the
// class of its continuum pair (integrals that break the declared symmetry).
__global__ void symmetry_check_kernel(const double *__restrict__ ttcc, const double *__restrict__ tctc,
                                      const double *__restrict__ h, int n_to, int n_co, int K,
                                      const int32_t *__restrict__ label_cls, const int32_t *__restrict__ co_irrep,
                                      int *__restrict__ flag) {
    const int jp = blockIdx.x * 32 + threadIdx.x, j = blockIdx.z;
    if (jp >= n_co) return;
    const int x = co_irrep[j] ^ co_irrep[jp];
    for (int k = blockIdx.y * 32 + threadIdx.y; k < K && k < (int)(blockIdx.y + 1) * 32; k += 8)
        if (label_cls[k] != x && label_value(ttcc, tctc, h, n_to, n_co, k, j, jp) != 0.0) atomicOr(flag, 1);
}

// FP64 TN GEMM with scatter: rows m = (jj, jjp) of a continuum rectangle,
// columns = the state pairs of every group pair merged into the block (each
// with its coefficient row and its own destination), K = Kpad labels.
constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(256)
expand_fp64_kernel(const XTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks,
                   const ExpCol *__restrict__ cols, int shard_r, int shard_n) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    if ((int)(blockIdx.x % (unsigned)shard_n) != shard_r) return;   // another shard's tile
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const XTask &T = tasks[ti];
    const double *__restrict__ P = T.P;
    const int32_t *__restrict__ perm = T.perm;
    const int Kpad = T.Kpad, n_co = T.n_co, cf = T.cf, cn = T.cn, cfp = T.cfp, cnp = T.cnp, N = T.N;
    const ExpCol *__restrict__ bc = cols + T.col0;
    const int lb = (int)(blockIdx.x - blk[ti]);
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t M = (int64_t)cn * cnp;
    const int64_t m0 = (int64_t)(lb % T.mtiles) * BM;
    const int n0 = (lb / T.mtiles) * BN;
    // loader: 64 rows x 16 k per operand, 4 doubles per thread
    const int lrow = tid / 4, lk = (tid % 4) * 4;
    const int64_t lm = m0 + lrow;
    const double *prow = nullptr;
    if (lm < M) {
        const int jj = (int)(lm / cnp), jjp = (int)(lm % cnp);
        prow = P + ((int64_t)(cf + jj) * n_co + (cfp + jjp)) * Kpad;
    }
    const int ln = n0 + lrow;
    const double *arow = ln < N ? bc[ln].arow : nullptr;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < Kpad; k0 += BK) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            As[lk + u][lrow] = prow ? __ldg(prow + k0 + lk + u) : 0.0;
            // the coefficient of the panel column: the label itself, or the
            // class's label list with orbital symmetry (-1: padding)
            const int lab = perm ? __ldg(perm + k0 + lk + u) : k0 + lk + u;
            Bs[lk + u][lrow] = (arow && lab >= 0) ? __ldg(arow + lab) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    // epilogue: H[(n, jj)][(n', jjp)] of the column's own matrix, and its mirror
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int t = n0 + tx * 4 + j;
        if (t >= N) continue;
        const ExpCol c = bc[t];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t m = m0 + ty * 4 + i;
            if (m >= M) continue;
            const int jj = (int)(m / cnp), jjp = (int)(m % cnp);
            const int64_t r = c.rbase + jj;
            const int64_t cc = c.cbase + jjp;
            if (c.same && r < cc) continue;
            c.H[r * c.ld + cc] = acc[i][j];
            if (r != cc) c.H[cc * c.ld + r] = acc[i][j];
        }
    }
}

}  // namespace

void build_panel(const double *ttcc, const double *tctc, const double *h, int n_to, int n_co, int Kc,
                 const int32_t *cls_labels, const int32_t *co_irrep, double *P, cudaStream_t s) {
    const dim3 grid((n_co + 31) / 32, Kc / 32, n_co), block(32, 8);
    panel_kernel<<<grid, block, 0, s>>>(ttcc, tctc, h, n_to, n_co, Kc, cls_labels, co_irrep, P);
}

void check_panel_symmetry(const double *ttcc, const double *tctc, const double *h, int n_to, int n_co, int K,
                          const int32_t *label_cls, const int32_t *co_irrep, int *flag, cudaStream_t s) {
    const dim3 grid((n_co + 31) / 32, (K + 31) / 32, n_co), block(32, 8);
    symmetry_check_kernel<<<grid, block, 0, s>>>(ttcc, tctc, h, n_to, n_co, K, label_cls, co_irrep, flag);
}

int expand_fp64_mtiles(int cn, int cnp) { return (int)(((int64_t)cn * cnp + BM - 1) / BM); }

int64_t blocks_expand_fp64(int cn, int cnp, int N) {
    if ((int64_t)cn * cnp == 0 || N == 0) return 0;
    return (int64_t)expand_fp64_mtiles(cn, cnp) * ((N + BN - 1) / BN);
}

int g_expand_fp64(const Grouped<XTask> &g, const ExpCol *cols, cudaStream_t s, int shard_r, int shard_n) {
    if (g.blocks <= 0) return 0;
    expand_fp64_kernel<<<(unsigned)g.blocks, 256, 0, s>>>(g.tasks, g.blk, g.n, cols, shard_r, shard_n);
    return 1;
}

}  // namespace hb
