// K3: expansion of the contracted prototype labels over the continuum orbitals
// (Eq. 7) for classes 1, 3, 5, 6, 7, double-precision path.
//
// With the contracted coefficients A[(n,n')][k] of K2 and the integral panel
// P[(j,j')][k] (one row per continuum pair, one column per label):
//   H~[(g n j), (g' n' j')] = sum_k P[(j,j')][k] * A[(n,n')][k]
// labels k: (jj'|rs) for r >= s, (jq|pj') for all (p, q), h_jj', delta_jj'.
// This file builds the panel (once, at staging) and runs the FP64 contraction
// with a scatter epilogue into the full symmetric continuum block.
#include "hb_internal.cuh"

namespace hb {

namespace {

// P[(j*n_co + jp)][k], tiles of 32 continuum orbitals jp x 32 labels k for one j,
// transposed through shared memory so reads and writes are both coalesced.
__global__ void panel_kernel(const double *__restrict__ ttcc, const double *__restrict__ tctc,
                             const double *__restrict__ h, int n_to, int n_co, int Kpad,
                             double *__restrict__ P) {
    __shared__ double tile[32][33];
    const int jp0 = blockIdx.x * 32, k0 = blockIdx.y * 32, j = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int Pt = n_to * (n_to + 1) / 2, nt2 = n_to * n_to, n_orb = n_to + n_co;
    const int64_t NTC = (int64_t)n_to * n_co, NCC = (int64_t)n_co * n_co;
    for (int r = ty; r < 32; r += 8) {
        const int k = k0 + r, jp = jp0 + tx;
        double v = 0.0;
        if (jp < n_co) {
            if (k < Pt) {
                v = ttcc[(int64_t)k * NCC + (int64_t)j * n_co + jp];
            } else if (k < Pt + nt2) {
                const int pq = k - Pt, p = pq / n_to, q = pq % n_to;
                v = tctc[((int64_t)q * n_co + j) * NTC + (int64_t)p * n_co + jp];
            } else if (k == Pt + nt2) {
                v = h[(int64_t)(n_to + j) * n_orb + n_to + jp];
            } else if (k == Pt + nt2 + 1) {
                v = (j == jp) ? 1.0 : 0.0;
            }
        }
        tile[r][tx] = v;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int jp = jp0 + r, k = k0 + tx;
        if (jp < n_co && k < Kpad) P[((int64_t)j * n_co + jp) * Kpad + k] = tile[tx][r];
    }
}

// FP64 TN GEMM with scatter: rows m = (jj, jjp) of the group pair's continuum
// block, columns t = state pair (n, n') from nn[], K = Kpad labels.
constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(256)
expand_fp64_kernel(const double *__restrict__ P, const double *__restrict__ A, const int32_t *__restrict__ nn,
                   int n_nn, int Kpad, int n_co, int cf, int cn, int cfp, int cnp, int64_t row_off,
                   int64_t col_off, int same_group, int64_t ld, double *__restrict__ H) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t M = (int64_t)cn * cnp;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    // loader: 64 rows x 16 k per operand, 4 doubles per thread
    const int lrow = tid / 4, lk = (tid % 4) * 4;
    const int64_t lm = m0 + lrow;
    const double *prow = nullptr;
    if (lm < M) {
        const int jj = (int)(lm / cnp), jjp = (int)(lm % cnp);
        prow = P + ((int64_t)(cf + jj) * n_co + (cfp + jjp)) * Kpad;
    }
    const int ln = n0 + lrow;
    const double *arow = ln < n_nn ? A + (int64_t)ln * Kpad : nullptr;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < Kpad; k0 += BK) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            As[lk + u][lrow] = prow ? __ldg(prow + k0 + lk + u) : 0.0;
            Bs[lk + u][lrow] = arow ? __ldg(arow + k0 + lk + u) : 0.0;
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
    // epilogue: H[(n, jj)][(n', jjp)] and its mirror
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t m = m0 + ty * 4 + i;
        if (m >= M) continue;
        const int jj = (int)(m / cnp), jjp = (int)(m % cnp);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int t = n0 + tx * 4 + j;
            if (t >= n_nn) continue;
            const int na = nn[2 * t], nb = nn[2 * t + 1];
            const int64_t r = row_off + (int64_t)na * cn + jj;
            const int64_t c = col_off + (int64_t)nb * cnp + jjp;
            if (same_group && r < c) continue;
            H[r * ld + c] = acc[i][j];
            if (r != c) H[c * ld + r] = acc[i][j];
        }
    }
}

}  // namespace

void build_panel(const double *ttcc, const double *tctc, const double *h, int n_to, int n_co, int Kpad,
                 double *P, cudaStream_t s) {
    const dim3 grid((n_co + 31) / 32, Kpad / 32, n_co), block(32, 8);
    panel_kernel<<<grid, block, 0, s>>>(ttcc, tctc, h, n_to, n_co, Kpad, P);
}

void expand_fp64(const double *P, const double *A, const int32_t *nn, int n_nn, int Kpad, int n_co, int cf,
                 int cn, int cfp, int cnp, int64_t row_off, int64_t col_off, int same_group, int64_t ld,
                 double *H, cudaStream_t s) {
    const int64_t M = (int64_t)cn * cnp;
    if (M == 0 || n_nn == 0) return;
    const dim3 grid((unsigned)((M + BM - 1) / BM), (n_nn + BN - 1) / BN);
    expand_fp64_kernel<<<grid, 256, 0, s>>>(P, A, nn, n_nn, Kpad, n_co, cf, cn, cfp, cnp, row_off, col_off,
                                            same_group, ld, H);
}

}  // namespace hb
