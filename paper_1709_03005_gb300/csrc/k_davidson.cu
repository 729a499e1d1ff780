// Block Davidson for the lowest k eigenpairs of the built matrix (Section
// 3.2.2 lists Davidson among the diagonalisers; the paper gives no details, so
// this is the standard block method):
//   basis V (orthonormal), AV = H V
//   Rayleigh-Ritz: T = V^T AV, T s = theta s, Ritz vectors x = V s, Ax = AV s
//   residuals r = Ax - theta x; stop when ||r_i|| <= tol for i < k
//   correction t_i = r_i / (H_ii - theta_i) (optionally times a learned factor)
//   t orthogonalised against V twice, then among itself (SVQB), appended
//   thick restart to the 2b lowest Ritz vectors when the basis is full.
// The products H V, the projection V^T AV, the Ritz combinations, residuals
// and the orthogonalisation run on the GPU in FP64 with fixed-order sums; only
// the small projected eigenproblem (at most a few hundred) is solved on the
// host (Householder tridiagonalisation and implicit QL).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "hb_api_internal.cuh"
#include "hb_davidson.cuh"

using namespace hb;

namespace {

// out[j][i] = beta * out[j][i] + sum_k A[i][k] B[j][k]  (i < M, j < N)
constexpr int GM = 64, GN = 32, GK = 16;
__global__ void __launch_bounds__(256)
gemm_nt_kernel(const double *__restrict__ A, int64_t lda, const double *__restrict__ B, int64_t ldb, int M, int N,
               int K, double *__restrict__ out, int64_t ldo, int beta) {
    __shared__ double As[GK][GM + 1];
    __shared__ double Bs[GK][GN + 1];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * GN;
    double acc[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int k0 = 0; k0 < K; k0 += GK) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = tid + u * 256, r = e / GK, kk = e % GK;
            const int gm = m0 + r, gk = k0 + kk;
            As[kk][r] = (gm < M && gk < K) ? __ldg(A + (int64_t)gm * lda + gk) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = tid + u * 256, r = e / GK, kk = e % GK;
            const int gn = n0 + r, gk = k0 + kk;
            Bs[kk][r] = (gn < N && gk < K) ? __ldg(B + (int64_t)gn * ldb + gk) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], b[2];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 2; ++j) b[j] = Bs[kk][tx * 2 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int gn = n0 + tx * 2 + j;
        if (gn >= N) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gm = m0 + ty * 4 + i;
            if (gm >= M) continue;
            double *o = out + (int64_t)gn * ldo + gm;
            *o = beta ? *o + acc[i][j] : acc[i][j];
        }
    }
}

// XT[l][j] = X[j][l] for l < rows, j < q: the vectors interleaved, so that
// one CSR column's q values are contiguous.  32 x 32 tiles through shared
// memory, both sides coalesced.
__global__ void interleave_kernel(const double *__restrict__ X, int64_t ldx, int64_t rows, int q,
                                  double *__restrict__ XT) {
    __shared__ double t[32][33];
    const int64_t l0 = (int64_t)blockIdx.x * 32;
    const int j0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = j0 + r;
        const int64_t l = l0 + threadIdx.x;
        t[r][threadIdx.x] = (j < q && l < rows) ? __ldg(X + (int64_t)j * ldx + l) : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t l = l0 + r;
        const int j = j0 + threadIdx.x;
        if (l < rows && j < q) XT[l * q + j] = t[threadIdx.x][r];
    }
}

// Y[j][l] += sum_p val[p] XT[col[p]][j] over CSR rows l (classes 2 and 8 of
// the matrix): one warp per row, lanes over vectors (in groups of 32),
// entries in order.  Each entry reads its column's vectors as one contiguous
// run of XT, so the warp's loads coalesce; the L2 block of an L2-heavy matrix
// (hundreds of millions of entries) streams once per product.
__global__ void spmm_csr_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                const double *__restrict__ val, int rows, const double *__restrict__ XT, int q,
                                double *__restrict__ Y, int64_t ldy) {
    const int lane = threadIdx.x & 31;
    const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (l >= rows) return;
    const int64_t b = rp[l], e = rp[l + 1];
    for (int j0 = 0; j0 < q; j0 += 32) {
        const int j = j0 + lane;
        double acc = 0.0;
        // 32 entries at a time: the warp loads their (column, value) pairs in
        // one coalesced read, then every lane walks them in order, taking each
        // pair from the lane that holds it; the gathers of one batch do not
        // depend on each other, so they are in flight together.
        for (int64_t p0 = b; p0 < e; p0 += 32) {
            const int64_t p = p0 + lane;
            const int c_mine = p < e ? __ldg(col + p) : 0;
            const double v_mine = p < e ? __ldg(val + p) : 0.0;
            const int cnt = (int)min((int64_t)32, e - p0);
#pragma unroll 8
            for (int t = 0; t < cnt; ++t) {
                const int c = __shfl_sync(0xffffffffu, c_mine, t);
                const double v = __shfl_sync(0xffffffffu, v_mine, t);
                if (j < q) acc = fma(v, __ldg(XT + (int64_t)c * q + j), acc);
            }
        }
        if (j < q) Y[(int64_t)j * ldy + l] += acc;
    }
}

// partial[c][a][b] = sum_{i in chunk c} X[a][i] Y[b][i]: one block per
// (chunk of kGramChunk entries, 32 x 32 tile of (a, b)); the rows of the tile
// pass through shared memory 64 entries at a time (coalesced along i), each
// thread keeps 4 outputs; fixed order, so the sums are deterministic.
constexpr int kGramChunk = 512;
constexpr int kGramTile = 32, kGramSub = 64;
__global__ void __launch_bounds__(256)
gram_partial_kernel(const double *__restrict__ X, int64_t ldx, int p, const double *__restrict__ Y, int64_t ldy, int q,
                    int64_t n, double *__restrict__ partial) {
    __shared__ double xs[kGramTile][kGramSub + 1], ys[kGramTile][kGramSub + 1];
    const int c = blockIdx.x;
    const int tiles_q = (q + kGramTile - 1) / kGramTile;
    const int a0 = (blockIdx.y / tiles_q) * kGramTile, b0 = (blockIdx.y % tiles_q) * kGramTile;
    const int64_t i0 = (int64_t)c * kGramChunk, i1 = (n < i0 + kGramChunk) ? n : i0 + kGramChunk;
    const int tid = threadIdx.x;
    const int ta = tid / 8, tb = (tid % 8) * 4;     // outputs (a0 + ta, b0 + tb .. tb + 3)
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t s0 = i0; s0 < i1; s0 += kGramSub) {
        __syncthreads();
        for (int e = tid; e < kGramTile * kGramSub; e += 256) {
            const int r = e / kGramSub, k = e % kGramSub;
            const int64_t i = s0 + k;
            xs[r][k] = (a0 + r < p && i < i1) ? __ldg(X + (int64_t)(a0 + r) * ldx + i) : 0.0;
            ys[r][k] = (b0 + r < q && i < i1) ? __ldg(Y + (int64_t)(b0 + r) * ldy + i) : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kGramSub; ++k) {
            const double x = xs[ta][k];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(x, ys[tb + u][k], acc[u]);
        }
    }
    const int a = a0 + ta;
    if (a < p)
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (b0 + tb + u < q) partial[(int64_t)c * p * q + (int64_t)a * q + b0 + tb + u] = acc[u];
}

// partial[c][a] = sum_{i in chunk c} X[a][i]^2: one block per (chunk, vector),
// each thread a strided share of the chunk, then a fixed-order tree over the
// block, so the sums are deterministic
__global__ void __launch_bounds__(256)
norms_partial_kernel(const double *__restrict__ X, int64_t ldx, int p, int64_t n, double *__restrict__ partial) {
    __shared__ double red[256];
    const int c = blockIdx.x, a = blockIdx.y;
    const int64_t i0 = (int64_t)c * kGramChunk, i1 = (n < i0 + kGramChunk) ? n : i0 + kGramChunk;
    double acc = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double x = __ldg(X + (int64_t)a * ldx + i);
        acc = fma(x, x, acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(int64_t)c * p + a] = red[0];
}

__global__ void reduce_kernel(const double *__restrict__ partial, int chunks, int nout, double *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nout) return;
    double acc = 0.0;
    for (int c = 0; c < chunks; ++c) acc += partial[(int64_t)c * nout + t];
    out[t] = acc;
}

// Y[j][i] = beta * Y[j][i] + scale * sum_a C[a][j] X[a][i]   (a < p, j < q), C on device [p][q];
// the coefficients pass through shared memory kCombineRows rows at a time.
constexpr int kCombineRows = 256;
__global__ void combine_kernel(const double *__restrict__ X, int64_t ldx, int p, const double *__restrict__ C, int q,
                               int64_t n, double *__restrict__ Y, int64_t ldy, double beta, double scale) {
    __shared__ double cs[kCombineRows * 16];
    const int j0 = blockIdx.y * 16;
    const int nq = min(16, q - j0);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double acc[16];
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) acc[jj] = 0.0;
    for (int a0 = 0; a0 < p; a0 += kCombineRows) {
        const int na = min(kCombineRows, p - a0);
        __syncthreads();
        for (int t = threadIdx.x; t < na * 16; t += blockDim.x) {
            const int a = t / 16, jj = t % 16;
            cs[t] = jj < nq ? scale * C[(int64_t)(a0 + a) * q + j0 + jj] : 0.0;
        }
        __syncthreads();
        if (i < n)
            for (int a = 0; a < na; ++a) {
                const double x = __ldg(X + (int64_t)(a0 + a) * ldx + i);
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) acc[jj] = fma(cs[a * 16 + jj], x, acc[jj]);
            }
    }
    if (i >= n) return;
#pragma unroll
    for (int jj = 0; jj < 16; ++jj)
        if (jj < nq) {
            double *y = Y + (int64_t)(j0 + jj) * ldy + i;
            *y = beta != 0.0 ? beta * *y + acc[jj] : acc[jj];
        }
}

// R[j] = AX[j] - theta_j X[j]
__global__ void residual_kernel(const double *__restrict__ AX, const double *__restrict__ X, int64_t ld,
                                const double *__restrict__ theta, int q, int64_t n, double *__restrict__ R) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n || j >= q) return;
    R[(int64_t)j * ld + i] = AX[(int64_t)j * ld + i] - theta[j] * X[(int64_t)j * ld + i];
}

// t[j] = w[i] * r[j] / (d_i - theta_j), with the denominator kept away from 0
__global__ void precond_kernel(const double *__restrict__ R, int64_t ld, const double *__restrict__ d,
                               const double *__restrict__ theta, const int32_t *__restrict__ which, int q, int64_t n,
                               const float *__restrict__ w, double *__restrict__ T, int64_t ldt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n || j >= q) return;
    const int src = which[j];
    double den = d[i] - theta[src];
    if (fabs(den) < 1e-4) den = den < 0 ? -1e-4 : 1e-4;
    double v = R[(int64_t)src * ld + i] / den;
    if (w) v *= (double)w[(int64_t)src * n + i];
    T[(int64_t)j * ldt + i] = v;
}

__global__ void diag_kernel(const double *__restrict__ Hcc, int64_t Dc, const int64_t *__restrict__ rp,
                            const int32_t *__restrict__ col, const double *__restrict__ val, int64_t nl,
                            double *__restrict__ d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Dc) {
        d[i] = Hcc[i * Dc + i];
    } else if (i < Dc + nl) {
        const int64_t l = i - Dc;
        double v = 0.0;
        for (int64_t p = rp[l]; p < rp[l + 1]; ++p)
            if (col[p] == (int32_t)l) { v = val[p]; break; }
        d[i] = v;
    }
}

__global__ void transpose_kernel(const double *__restrict__ in, int64_t rows, int64_t cols, double *__restrict__ out) {
    __shared__ double tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < rows && c < cols) ? in[r * cols + c] : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[c * rows + r] = tile[threadIdx.x][k];
    }
}

__global__ void unit_vectors_kernel(double *V, int64_t ld, const int32_t *idx, int q, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n || j >= q) return;
    V[(int64_t)j * ld + i] = (i == idx[j]) ? 1.0 : 0.0;
}

// evecs[i][j] = X[j][i] (row-major dim x k)
__global__ void export_kernel(const double *__restrict__ X, int64_t ld, int k, int64_t n, double *__restrict__ E) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n || j >= k) return;
    E[i * k + j] = X[(int64_t)j * ld + i];
}

__global__ void import_kernel(const double *__restrict__ E, int k, int64_t n, double *__restrict__ X, int64_t ld) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n || j >= k) return;
    X[(int64_t)j * ld + i] = E[i * k + j];
}

}  // namespace

// The diagonal of H from the built blocks into w->d.
void hb::fill_diag(hb_ctx *ctx, const hb_blocks *H, DiagWork *w, cudaStream_t s) {
    diag_kernel<<<(unsigned)((ctx->dim + 255) / 256), 256, 0, s>>>(H->Hcc, ctx->Dc, H->l2_row_ptr, H->l2_col,
                                                                    H->l2_val, ctx->n_l2, w->d);
}

// ------------------------------------------------------------ host solver
// Symmetric eigensolver for the small projected matrix: Householder reduction
// to tridiagonal form, then the implicit-shift QL iteration on the tridiagonal
// matrix with the transformations accumulated (the classical two-phase method,
// as in Golub & Van Loan and Wilkinson & Reinsch).  A is n x n row-major; on
// return w holds the eigenvalues ascending and column j of V (V[i*n + j]) the
// eigenvector of w[j].
// ----------------------------------------- small dense symmetric eigensolver
// All eigenvalues and the eigenvectors of the nvec lowest of a symmetric n x n
// matrix (the Rayleigh-Ritz and Gram matrices of the solver, n up to about a
// thousand), on the host:
//   1. Householder reduction to tridiagonal form, Q^T A Q = T (Golub & Van
//      Loan, Alg. 8.3.1), with the symmetric rank-2 update of the trailing
//      block done row by row;
//   2. the eigenvalues of T by implicit QR steps with the Wilkinson shift
//      (Golub & Van Loan, Alg. 8.3.3), without accumulating vectors;
//   3. each wanted eigenvector of T by inverse iteration (three solves of the
//      shifted tridiagonal system with partial pivoting), orthogonalised
//      against the vectors of the same cluster;
//   4. the back-transformation x = Q y with the stored reflectors.
// w: ascending eigenvalues [n]; V: [n][nvec], column c is the c-th vector.
namespace {

struct Tridiag {
    std::vector<double> d, e;          // diagonal [n], off-diagonal [n-1]
    std::vector<double> vs, beta;      // reflector k: vs[k][k+1..n), beta[k]
};

Tridiag tridiagonalize(int n, std::vector<double> &A) {
    Tridiag t;
    t.d.assign(n, 0.0);
    t.e.assign(n > 1 ? n - 1 : 0, 0.0);
    t.vs.assign((size_t)n * n, 0.0);
    t.beta.assign(n, 0.0);
    std::vector<double> p(n), pn(n), wv(n), col(n);
    std::vector<char> ready(n, 0), skip(n, 0);
    int have_p = 0;
    // reflector k from x = column k below the diagonal (x[i] for i > k):
    // v = x - alpha e_{k+1}, alpha = -sign(x_{k+1}) |x|, beta = 2 / v.v
    auto reflector = [&](int k, const double *x) {
        double xn = 0.0;
        for (int i = k + 1; i < n; ++i) xn += x[i] * x[i];
        xn = std::sqrt(xn);
        ready[k] = 1;
        if (xn == 0.0) { t.e[k] = 0.0; skip[k] = 1; return; }
        const double alpha = x[k + 1] >= 0.0 ? -xn : xn;
        double *v = &t.vs[(size_t)k * n];
        for (int i = k + 1; i < n; ++i) v[i] = x[i];
        v[k + 1] -= alpha;
        double vv = 0.0;
        for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
        t.e[k] = alpha;
        if (vv == 0.0) { skip[k] = 1; return; }
        t.beta[k] = 2.0 / vv;
    };
    // One parallel region for the whole reduction on the large projected
    // matrices.  Step k: p = beta A22 v, w = p - (beta/2)(p.v) v,
    // A22 -= v w^T + w v^T.  The update of column k+1 is formed first (O(n)),
    // which gives reflector k+1, so one pass over the trailing block both
    // applies step k and computes the product A22 v of step k+1 (the look-ahead
    // column uses the same expression as the pass, so the values agree).
#pragma omp parallel if (n > 192)
    for (int k = 0; k + 2 < n; ++k) {
#pragma omp single
        {
            if (!ready[k]) {
                for (int i = k + 1; i < n; ++i) col[i] = A[(size_t)i * n + k];
                reflector(k, col.data());
            }
        }
        if (skip[k]) {
#pragma omp single
            have_p = 0;
            continue;
        }
        const double *v = &t.vs[(size_t)k * n];
        const double bk = t.beta[k];
        if (!have_p) {
#pragma omp for schedule(static)
            for (int i = k + 1; i < n; ++i) {
                const double *row = &A[(size_t)i * n];
                double acc = 0.0;
                for (int j = k + 1; j < n; ++j) acc += row[j] * v[j];
                p[i] = bk * acc;
            }
        }
#pragma omp single
        {
            double pv = 0.0;
            for (int i = k + 1; i < n; ++i) pv += p[i] * v[i];
            for (int i = k + 1; i < n; ++i) wv[i] = p[i] - 0.5 * bk * pv * v[i];
            // look-ahead: column k+1 after this step's update, and its reflector
            if (k + 3 < n) {
                const int c = k + 1;
                for (int i = c + 1; i < n; ++i) col[i] = A[(size_t)i * n + c] - (v[i] * wv[c] + wv[i] * v[c]);
                reflector(c, col.data());
            }
        }
        const int nx = k + 1;
        const bool next = k + 3 < n && !skip[nx];
        const double *vn = &t.vs[(size_t)nx * n];
        const double bn = t.beta[nx];
#pragma omp for schedule(static)
        for (int i = k + 1; i < n; ++i) {
            double *row = &A[(size_t)i * n];
            const double vi = v[i], wi = wv[i];
            double acc = 0.0;
            if (next && i > nx) {
                row[nx] -= vi * wv[nx] + wi * v[nx];
                for (int j = nx + 1; j < n; ++j) {
                    row[j] -= vi * wv[j] + wi * v[j];
                    acc += row[j] * vn[j];
                }
                pn[i] = bn * acc;
            } else {
                for (int j = k + 1; j < n; ++j) row[j] -= vi * wv[j] + wi * v[j];
            }
        }
#pragma omp single
        {
            have_p = next ? 1 : 0;
            if (next) p.swap(pn);
        }
    }
    for (int i = 0; i < n; ++i) t.d[i] = A[(size_t)i * n + i];
    if (n >= 2) t.e[n - 2] = A[(size_t)(n - 1) * n + (n - 2)];
    return t;
}

// All eigenvalues of T by implicit symmetric QR steps with the Wilkinson
// shift and deflation (Golub & Van Loan, Alg. 8.3.3): each step chases the
// bulge of one Givens rotation G^T T G down the unreduced block [p, q].
std::vector<double> tridiag_eigenvalues(const Tridiag &t) {
    const int n = (int)t.d.size();
    std::vector<double> a(t.d), b(t.e);
    b.push_back(0.0);
    int q = n - 1;
    int guard = 0;
    while (q > 0 && guard < 60 * n) {
        // deflate negligible couplings at the bottom
        if (std::fabs(b[q - 1]) <= 2.2e-16 * (std::fabs(a[q - 1]) + std::fabs(a[q]))) {
            b[q - 1] = 0.0;
            --q;
            continue;
        }
        int p = q - 1;
        while (p > 0 && std::fabs(b[p - 1]) > 2.2e-16 * (std::fabs(a[p - 1]) + std::fabs(a[p]))) --p;
        if (p > 0) b[p - 1] = 0.0;
        // Wilkinson shift from the trailing 2 x 2 block
        const double dlt = 0.5 * (a[q - 1] - a[q]);
        const double bq = b[q - 1];
        const double den = dlt + (dlt >= 0.0 ? std::hypot(dlt, bq) : -std::hypot(dlt, bq));
        const double mu = den != 0.0 ? a[q] - bq * bq / den : a[q] - std::fabs(bq);
        double x = a[p] - mu, z = b[p];
        for (int k = p; k < q; ++k) {
            const double r = std::hypot(x, z);
            const double c = r != 0.0 ? x / r : 1.0, s = r != 0.0 ? -z / r : 0.0;
            if (k > p) b[k - 1] = r;
            const double ak = a[k], ak1 = a[k + 1], bk = b[k];
            a[k] = c * c * ak - 2.0 * c * s * bk + s * s * ak1;
            a[k + 1] = s * s * ak + 2.0 * c * s * bk + c * c * ak1;
            b[k] = c * s * (ak - ak1) + (c * c - s * s) * bk;
            if (k + 1 < q) {
                x = b[k];
                z = -s * b[k + 1];
                b[k + 1] = c * b[k + 1];
            }
        }
        ++guard;
    }
    std::sort(a.begin(), a.end());
    return a;
}

// The nvec lowest eigenvalues of T by bisection on Sturm counts (Golub & Van
// Loan, Sec. 8.4.1): the number of eigenvalues below x is the number of
// negative pivots of the LDL^T factorisation of T - x I.  Each eigenvalue is
// bracketed from the Gershgorin interval independently, so they are found in
// parallel, to a width of a few units in the last place.
std::vector<double> tridiag_lowest(const Tridiag &t, int nvec) {
    const int n = (int)t.d.size();
    double lo = 0.0, hi = 0.0;
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? std::fabs(t.e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(t.e[i]) : 0.0);
        lo = i ? std::min(lo, t.d[i] - r) : t.d[i] - r;
        hi = i ? std::max(hi, t.d[i] + r) : t.d[i] + r;
    }
    const double pad = 2.2e-16 * std::max(std::fabs(lo), std::fabs(hi)) + 1e-300;
    lo -= pad;
    hi += pad;
    std::vector<double> e2(n > 1 ? n - 1 : 0);
    for (int i = 0; i + 1 < n; ++i) e2[i] = t.e[i] * t.e[i];
    const double tiny = 1e-300 + 2.2e-16 * std::max(std::fabs(lo), std::fabs(hi)) * 1e-10;
    auto below = [&](double x) {
        int c = 0;
        double q = t.d[0] - x;
        if (q < 0.0) ++c;
        for (int i = 1; i < n; ++i) {
            if (q == 0.0) q = -tiny;
            q = t.d[i] - x - e2[i - 1] / q;
            if (q < 0.0) ++c;
        }
        return c;
    };
    std::vector<double> w(nvec);
#pragma omp parallel for schedule(dynamic, 4) if ((int64_t)nvec * n > 20000)
    for (int j = 0; j < nvec; ++j) {
        double a = lo, b = hi;
        for (int it = 0; it < 2100; ++it) {
            const double mid = 0.5 * (a + b);
            if (mid <= a || mid >= b || b - a <= 2.0 * 2.2e-16 * std::max(std::fabs(a), std::fabs(b))) break;
            if (below(mid) > j) b = mid;
            else a = mid;
        }
        w[j] = 0.5 * (a + b);
    }
    return w;
}

// eigenvector of T for the eigenvalue lam by inverse iteration; the vectors
// in `cluster` (unit, orthogonal) are projected out after every solve
void tridiag_vector(const Tridiag &t, double lam, double tnorm, int seed, const std::vector<const double *> &cluster,
                    double *y) {
    const int n = (int)t.d.size();
    if (n == 1) { y[0] = 1.0; return; }
    // shifted matrix, perturbed off the eigenvalue so the factors are finite
    const double shift = lam + 4.0 * 2.2e-16 * tnorm;
    // LU with partial pivoting of the tridiagonal T - shift I:
    // U has diagonal u0, superdiagonals u1, u2; L multipliers mul, row swaps piv
    std::vector<double> u0(n), u1(n), u2(n), mul(n);
    std::vector<char> piv(n);
    {
        double a = t.d[0] - shift, b = t.e[0], c = 0.0;
        for (int i = 0; i < n - 1; ++i) {
            const double lo = t.e[i];                   // subdiagonal entry of row i + 1
            const double na = t.d[i + 1] - shift;
            const double nb = i + 1 < n - 1 ? t.e[i + 1] : 0.0;
            if (std::fabs(a) >= std::fabs(lo)) {
                piv[i] = 0;
                const double m = a != 0.0 ? lo / a : 0.0;
                mul[i] = m;
                u0[i] = a; u1[i] = b; u2[i] = c;
                a = na - m * b;
                b = nb - m * c;
                c = 0.0;
            } else {
                piv[i] = 1;
                const double m = a / lo;
                mul[i] = m;
                u0[i] = lo; u1[i] = na; u2[i] = nb;
                a = b - m * na;
                b = c - m * nb;
                c = 0.0;
            }
        }
        u0[n - 1] = a;
    }
    const double tiny = 2.2e-16 * tnorm + 1e-300;
    for (int i = 0; i < n; ++i)
        if (std::fabs(u0[i]) < tiny) u0[i] = u0[i] < 0.0 ? -tiny : tiny;
    // deterministic start vector
    uint64_t r = 0x9e3779b97f4a7c15ull * (uint64_t)(seed + 1);
    for (int i = 0; i < n; ++i) {
        r ^= r >> 12; r ^= r << 25; r ^= r >> 27;
        y[i] = 0.5 + (double)((r * 2685821657736338717ull) >> 11) * (1.0 / 9007199254740992.0);
    }
    // Two Gram-Schmidt passes: in a large cluster of nearly equal eigenvalues
    // the solve returns y almost inside the span of the earlier vectors, and
    // one pass leaves the rounding of that large part in the small remainder
    // (with fused multiply-adds that reached 1e-9 of orthogonality on the Gram
    // matrices of the block orthonormalisation); the second pass removes it.
    auto orth_normalise = [&]() {
        for (int pass = 0; pass < 2; ++pass)
            for (const double *q : cluster) {
                double dot = 0.0;
                for (int i = 0; i < n; ++i) dot += q[i] * y[i];
                for (int i = 0; i < n; ++i) y[i] -= dot * q[i];
            }
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) nrm += y[i] * y[i];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) { y[seed % n] = 1.0; nrm = 1.0; }
        for (int i = 0; i < n; ++i) y[i] /= nrm;
    };
    orth_normalise();
    for (int it = 0; it < 3; ++it) {
        // forward: apply the row swaps and multipliers
        for (int i = 0; i < n - 1; ++i) {
            if (piv[i]) std::swap(y[i], y[i + 1]);
            y[i + 1] -= mul[i] * y[i];
        }
        // back substitution with U (bandwidth 3)
        for (int i = n - 1; i >= 0; --i) {
            double s = y[i];
            if (i + 1 < n) s -= u1[i] * y[i + 1];
            if (i + 2 < n) s -= u2[i] * y[i + 2];
            y[i] = s / u0[i];
        }
        orth_normalise();
    }
}

}  // namespace

void hb::small_eigh(int n, std::vector<double> A, std::vector<double> &w, std::vector<double> &V, int nvec) {
    if (nvec < 0 || nvec > n) nvec = n;
    w.assign(n, 0.0);
    V.assign((size_t)n * std::max(nvec, 1), 0.0);
    if (n == 0) return;
    if (n == 1) { w[0] = A[0]; if (nvec) V[0] = 1.0; return; }
    Tridiag t = tridiagonalize(n, A);
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? std::fabs(t.e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(t.e[i]) : 0.0);
        tnorm = std::max(tnorm, std::fabs(t.d[i]) + r);
    }
    if (n >= 256 && 2 * nvec < n) {
        // the wanted lowest by bisection (cheaper than all of them by QR on
        // the large projected matrices); w then holds those nvec
        const std::vector<double> low = tridiag_lowest(t, nvec);
        std::copy(low.begin(), low.end(), w.begin());
        w.resize(nvec);
    } else {
        w = tridiag_eigenvalues(t);
    }
    // vectors of the nvec lowest, each orthogonalised against the earlier
    // vectors whose eigenvalues lie within gap; runs of eigenvalues whose
    // neighbours are closer than gap are independent and run in parallel
    const double gap = 1e-3 * std::max(tnorm, 1e-300);
    std::vector<int> first;
    for (int c = 0; c < nvec; ++c)
        if (c == 0 || w[c] - w[c - 1] > gap) first.push_back(c);
    first.push_back(nvec);
    std::vector<double> Y((size_t)std::max(nvec, 1) * n);
    const int n_runs = (int)first.size() - 1;
#pragma omp parallel for schedule(dynamic, 1) if ((int64_t)nvec * n > 65536)
    for (int cl = 0; cl < n_runs; ++cl) {
        for (int c = first[cl]; c < first[cl + 1]; ++c) {
            std::vector<const double *> cluster;
            for (int c2 = c - 1; c2 >= first[cl] && w[c] - w[c2] <= gap; --c2) cluster.push_back(&Y[(size_t)c2 * n]);
            tridiag_vector(t, w[c], tnorm, c, cluster, &Y[(size_t)c * n]);
        }
    }
    // back-transformation x = H_0 H_1 ... y (reflectors applied last to first)
#pragma omp parallel for schedule(static) if ((int64_t)nvec * n > 65536)
    for (int c = 0; c < nvec; ++c) {
        double *y = &Y[(size_t)c * n];
        for (int k = n - 3; k >= 0; --k) {
            if (t.beta[k] == 0.0) continue;
            const double *v = &t.vs[(size_t)k * n];
            double dot = 0.0;
            for (int i = k + 1; i < n; ++i) dot += v[i] * y[i];
            dot *= t.beta[k];
            for (int i = k + 1; i < n; ++i) y[i] -= dot * v[i];
        }
        for (int i = 0; i < n; ++i) V[(size_t)i * nvec + c] = y[i];
    }
}

// test entry: the nvec lowest eigenpairs (w [nvec], V [n][nvec])
extern "C" int hb_test_symeig(int n, const double *A, int nvec, double *w, double *V) {
    std::vector<double> a(A, A + (size_t)n * n), ww, vv;
    hb::small_eigh(n, a, ww, vv, nvec);
    std::memcpy(w, ww.data(), sizeof(double) * nvec);
    std::memcpy(V, vv.data(), sizeof(double) * (size_t)n * nvec);
    return 0;
}

// ------------------------------------------------------------ the solver
namespace {

struct Ops {
    hb_ctx *ctx;
    const hb_blocks *H;
    cudaStream_t s;
    int64_t n, Dc, nl;
    DiagWork *w;
    bool force_fp64 = false;   // products in FP64 even when the tensor-core slices exist
    int launches = 0;
    double ms_gram = 0.0, ms_combine = 0.0, ms_eigh = 0.0;
    double proj_flops = 0.0;   // FP64 flops of gram, norms2, combine and project_out
    static double now_ms() {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
    }

    // Y[0:q] = H X[0:q], vectors stored as rows of length ld
    void matvec(const double *X, double *Y, int q, int64_t ld) {
        if (q <= 0) return;
        if (w->tc && !force_fp64) {
            // split-bf16 tensor-core products: Y_c = [Hcc | Hlc^T] X, Y_l = Hlc X_c
            // (+ the L2 block in FP64 below)
            dense_operand_fill(w->Xs, w->S, X, ld, (int)n, nullptr, 0, 0, q, s);
            ++launches;
            if (Dc > 0) launches += dense_split_gemm(w->S, w->A1, Dc, w->Xs, q, w->A1.planes, w->part, Y, ld, w->err, s);
            if (nl > 0) {
                if (Dc > 0) {
                    launches += dense_split_gemm(w->S, w->A2, nl, w->Xs, q, w->A2.planes, w->part, Y + Dc, ld, w->err, s);
                } else {
                    for (int j = 0; j < q; ++j) cudaMemsetAsync(Y + (int64_t)j * ld, 0, sizeof(double) * nl, s);
                }
                l2_product(X, Y, q, ld);
            }
            return;
        }
        if (Dc > 0) {
            dim3 g((unsigned)((Dc + GM - 1) / GM), (q + GN - 1) / GN);
            gemm_nt_kernel<<<g, 256, 0, s>>>(H->Hcc, Dc, X, ld, (int)Dc, q, (int)Dc, Y, ld, 0);
            ++launches;
            if (nl > 0) {
                gemm_nt_kernel<<<g, 256, 0, s>>>(w->HlcT, nl, X + Dc, ld, (int)Dc, q, (int)nl, Y, ld, 1);
                ++launches;
            }
        }
        if (nl > 0) {
            dim3 g((unsigned)((nl + GM - 1) / GM), (q + GN - 1) / GN);
            if (Dc > 0) {
                gemm_nt_kernel<<<g, 256, 0, s>>>(H->Hlc, Dc, X, ld, (int)nl, q, (int)Dc, Y + Dc, ld, 0);
                ++launches;
            } else {
                for (int j = 0; j < q; ++j) cudaMemsetAsync(Y + (int64_t)j * ld, 0, sizeof(double) * nl, s);
            }
            l2_product(X, Y, q, ld);
        }
    }

    // Y_l += (L2 block) X_l for the q vectors: interleave the L2 part of the
    // vectors, then the CSR product
    void l2_product(const double *X, double *Y, int q, int64_t ld) {
        for (int j0 = 0; j0 < q; j0 += w->mmax) {
            const int qq = std::min(q - j0, w->mmax);
            dim3 gi((unsigned)((nl + 31) / 32), (unsigned)((qq + 31) / 32));
            interleave_kernel<<<gi, dim3(32, 8), 0, s>>>(X + (int64_t)j0 * ld + Dc, ld, nl, qq, w->XT);
            spmm_csr_kernel<<<(unsigned)((nl + 7) / 8), 256, 0, s>>>(H->l2_row_ptr, H->l2_col, H->l2_val, (int)nl,
                                                                     w->XT, qq, Y + (int64_t)j0 * ld + Dc, ld);
            launches += 2;
        }
    }

    // G[a][b] = X[a] . Y[b] on the host (p x q)
    void gram(const double *X, int p, const double *Y, int q, int64_t ld, std::vector<double> &G) {
        const double t0 = now_ms();
        const int chunks = (int)((n + kGramChunk - 1) / kGramChunk);
        dim3 g(chunks, ((p + kGramTile - 1) / kGramTile) * ((q + kGramTile - 1) / kGramTile));
        gram_partial_kernel<<<g, 256, 0, s>>>(X, ld, p, Y, ld, q, n, w->partial);
        reduce_kernel<<<(p * q + 255) / 256, 256, 0, s>>>(w->partial, chunks, p * q, w->small);
        launches += 2;
        proj_flops += 2.0 * p * q * (double)n;
        G.resize((size_t)p * q);
        cudaMemcpyAsync(G.data(), w->small, sizeof(double) * p * q, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        ms_gram += now_ms() - t0;
    }

    // r2[a] = |X[a]|^2 on the host (p values)
    void norms2(const double *X, int p, int64_t ld, std::vector<double> &r2) {
        const double t0 = now_ms();
        const int chunks = (int)((n + kGramChunk - 1) / kGramChunk);
        norms_partial_kernel<<<dim3(chunks, p), 256, 0, s>>>(X, ld, p, n, w->partial);
        reduce_kernel<<<(p + 255) / 256, 256, 0, s>>>(w->partial, chunks, p, w->small);
        launches += 2;
        proj_flops += 2.0 * p * (double)n;
        r2.resize((size_t)p);
        cudaMemcpyAsync(r2.data(), w->small, sizeof(double) * p, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        ms_gram += now_ms() - t0;
    }

    void eigh(int m, std::vector<double> &A, std::vector<double> &wv, std::vector<double> &V, int nvec) {
        const double t0 = now_ms();
        small_eigh(m, A, wv, V, nvec);
        ms_eigh += now_ms() - t0;
    }

    // Y[0:q] = beta Y + X[0:p]^T C, C host [p][q]
    void combine(const double *X, int p, const std::vector<double> &C, int q, double *Y, int64_t ld, double beta) {
        const double t0 = now_ms();
        cudaMemcpyAsync(w->small, C.data(), sizeof(double) * p * q, cudaMemcpyHostToDevice, s);
        dim3 g((unsigned)((n + 255) / 256), (q + 15) / 16);
        combine_kernel<<<g, 256, 0, s>>>(X, ld, p, w->small, q, n, Y, ld, beta, 1.0);
        ++launches;
        proj_flops += 2.0 * p * q * (double)n;
        // no wait: the next upload into w->small is ordered after this kernel
        // on the stream, and the pageable source is staged before the copy call returns
        ms_combine += now_ms() - t0;
    }

    // Y[0:q] -= X[0:p]^T (X[0:p] Y[0:q]^T): one projection pass, all on the device
    void project_out(const double *X, int p, double *Y, int q, int64_t ld) {
        if (p <= 0 || q <= 0) return;
        const double t0 = now_ms();
        const int chunks = (int)((n + kGramChunk - 1) / kGramChunk);
        dim3 g(chunks, ((p + kGramTile - 1) / kGramTile) * ((q + kGramTile - 1) / kGramTile));
        gram_partial_kernel<<<g, 256, 0, s>>>(X, ld, p, Y, ld, q, n, w->partial);
        reduce_kernel<<<(p * q + 255) / 256, 256, 0, s>>>(w->partial, chunks, p * q, w->proj);
        dim3 g2((unsigned)((n + 255) / 256), (q + 15) / 16);
        combine_kernel<<<g2, 256, 0, s>>>(X, ld, p, w->proj, q, n, Y, ld, 1.0, -1.0);
        launches += 3;
        proj_flops += 4.0 * p * q * (double)n;
        ms_gram += now_ms() - t0;
    }
};

}  // namespace

static int diag_fail(hb_ctx *ctx, int code, const std::string &m) {
    ctx->err = m;
    return code;
}

static void release_tensor_products(hb_ctx *ctx, DiagWork *w) {
    dense_operand_free(ctx, &w->A1);
    dense_operand_free(ctx, &w->A2);
    dense_operand_free(ctx, &w->Xs);
    dfree(ctx, w->part);
    dfree(ctx, w->err);
    w->part = nullptr;
    w->err = nullptr;
    w->tc = false;
}

// Slices of [Hcc | Hlc^T] and of Hlc (fixed during the solve), the vector
// slice buffer for up to mmax vectors and the split-K scratch.
static int setup_tensor_products(hb_ctx *ctx, const hb_blocks *H, DiagWork *w, int mmax, cudaStream_t s) {
    release_tensor_products(ctx, w);
    const int64_t n = ctx->dim, Dc = ctx->Dc, nl = ctx->n_l2;
    const int S = ctx->split_slices >= 2 && ctx->split_slices <= 6 ? ctx->split_slices : 6;
    w->S = S;
    std::string err;
    const int K1 = (int)((n + 63) / 64 * 64), K2 = (int)((Dc + 63) / 64 * 64);
    int rc = dense_operand_alloc(ctx, S, mmax, K1, &w->Xs, &err);
    if (rc == HB_OK && Dc > 0) rc = dense_operand_alloc(ctx, S, Dc, K1, &w->A1, &err);
    if (rc == HB_OK && Dc > 0 && nl > 0) rc = dense_operand_alloc(ctx, S, nl, K2, &w->A2, &err);
    size_t part = 1;
    int per = 0;
    if (Dc > 0) part = std::max(part, (size_t)dense_splits(Dc, 1, K1 / 64, &per) * mmax * Dc);
    if (Dc > 0 && nl > 0) part = std::max(part, (size_t)dense_splits(nl, 1, K2 / 64, &per) * mmax * nl);
    cudaError_t e = cudaSuccess;
    if (rc == HB_OK) e = dmalloc_n(ctx, &w->part, part);
    if (rc == HB_OK && e == cudaSuccess) e = dmalloc_n(ctx, &w->err, 1);
    if (rc == HB_OK && e == cudaSuccess) e = cudaMemsetAsync(w->err, 0, sizeof(int), s);
    if (rc == HB_OK && e != cudaSuccess) {
        rc = HB_ERR_OOM;
        err = std::string("Davidson tensor-core scratch: ") + cudaGetErrorString(e);
    }
    if (rc != HB_OK) {
        release_tensor_products(ctx, w);
        return diag_fail(ctx, rc, err);
    }
    if (Dc > 0) dense_operand_fill(w->A1, S, H->Hcc, Dc, (int)Dc, nl > 0 ? w->HlcT : nullptr, nl, (int)nl, Dc, s);
    if (Dc > 0 && nl > 0) dense_operand_fill(w->A2, S, H->Hlc, Dc, (int)Dc, nullptr, 0, 0, nl, s);
    w->tc = true;
    return HB_OK;
}

// Device bytes a solve for k eigenpairs takes from the context's memory (the
// allocations of ensure_diag_work, of the interleaved vectors and the class-4
// transpose, of the tensor-core slices, and of the learned factors), each
// rounded as the context's allocator rounds it.
int64_t hb::diag_workspace_bytes(const hb_ctx *ctx, int k, int precond) {
    auto r = [](double b) { return (int64_t)((std::max<double>(b, 1.0) + 255.0) / 256.0) * 256; };
    const int64_t n = ctx->dim, Dc = ctx->Dc, nl = ctx->n_l2;
    if (n < 1 || k < 1) return 0;
    const int b = (int)std::min<int64_t>(n, k + std::max(4, std::min(16, k / 2)));
    const int mmax = (int)std::min<int64_t>(n, (int64_t)ctx->diag_basis * b);
    const int64_t chunks = (n + kGramChunk - 1) / kGramChunk;
    int64_t t = 5 * r(8.0 * mmax * n) + r(8.0 * n) + r(8.0 * chunks * mmax * mmax) + 2 * r(8.0 * mmax * mmax) +
                r(8.0 * mmax) + r(4.0 * mmax);
    if (nl > 0) t += r(8.0 * nl * mmax);
    if (Dc > 0 && nl > 0) t += r(8.0 * Dc * nl);
    if (precond & HB_DIAG_TENSOR) {
        const int S = ctx->split_slices >= 2 && ctx->split_slices <= 6 ? ctx->split_slices : 6;
        const int64_t K1 = (n + 63) / 64 * 64, K2 = (Dc + 63) / 64 * 64;
        t += r(2.0 * S * K1 * mmax);
        if (Dc > 0) t += r(2.0 * S * K1 * Dc);
        if (Dc > 0 && nl > 0) t += r(2.0 * S * K2 * nl);
        size_t part = 1;
        int per = 0;
        if (Dc > 0) part = std::max(part, (size_t)dense_splits(Dc, 1, (int)(K1 / 64), &per) * mmax * Dc);
        if (Dc > 0 && nl > 0) part = std::max(part, (size_t)dense_splits(nl, 1, (int)(K2 / 64), &per) * mmax * nl);
        t += r(8.0 * part) + r(4.0);
    }
    if ((precond & 0xff) == HB_PRECOND_MLP) t += r(16.0 * n) + r(4.0 * b * n);
    return t;
}

int hb::ensure_diag_work(hb_ctx *ctx, const hb_blocks *H, int mmax, cudaStream_t s) {
    DiagWork *w = (DiagWork *)ctx->diag;
    const int64_t n = ctx->dim;
    if (!w) {
        w = new DiagWork();
        ctx->diag = w;
    }
    if (w->mmax < mmax || w->n != n) {
        auto fr = [&](void *p) { dfree(ctx, p); };
        fr(w->V); fr(w->AV); fr(w->X); fr(w->AX); fr(w->W2); fr(w->d); fr(w->partial); fr(w->small); fr(w->theta);
        fr(w->idx); fr(w->proj); fr(w->XT);
        w->V = w->AV = w->X = w->AX = w->W2 = w->d = w->partial = w->small = w->theta = w->proj = w->XT = nullptr;
        w->idx = nullptr;
        w->XT_rows = 0;
        const size_t vec = (size_t)mmax * n;
        cudaError_t e = dmalloc_n(ctx, &w->V, vec);
        if (e == cudaSuccess) e = dmalloc_n(ctx, &w->AV, vec);
        if (e == cudaSuccess) e = dmalloc_n(ctx, &w->X, vec);
        if (e == cudaSuccess) e = dmalloc_n(ctx, &w->AX, vec);
        if (e == cudaSuccess) e = dmalloc_n(ctx, &w->W2, vec);
        if (e == cudaSuccess) e = dmalloc_n(ctx, &w->d, (size_t)n);
        const int chunks = (int)((n + kGramChunk - 1) / kGramChunk);
        if (e == cudaSuccess) e = dmalloc_n(ctx, &w->partial, (size_t)chunks * mmax * mmax);
        if (e == cudaSuccess) e = dmalloc_n(ctx, &w->small, (size_t)mmax * mmax);
        if (e == cudaSuccess) e = dmalloc_n(ctx, &w->proj, (size_t)mmax * mmax);
        if (e == cudaSuccess) e = dmalloc_n(ctx, &w->theta, (size_t)mmax);
        if (e == cudaSuccess) e = dmalloc_n(ctx, &w->idx, (size_t)mmax);
        if (e != cudaSuccess) return diag_fail(ctx, HB_ERR_OOM, std::string("Davidson workspace: ") + cudaGetErrorString(e));
        w->mmax = mmax;
        w->n = n;
    }
    if (ctx->n_l2 > 0 && w->XT_rows < (int64_t)ctx->n_l2 * w->mmax) {
        dfree(ctx, w->XT);
        w->XT = nullptr;
        w->XT_rows = 0;
        cudaError_t e = dmalloc_n(ctx, &w->XT, (size_t)ctx->n_l2 * w->mmax);
        if (e != cudaSuccess) return diag_fail(ctx, HB_ERR_OOM, "Davidson interleaved-vector buffer");
        w->XT_rows = (int64_t)ctx->n_l2 * w->mmax;
    }
    if (ctx->Dc > 0 && ctx->n_l2 > 0 && (!w->HlcT || w->HlcT_src != H->Hlc)) {
        if (!w->HlcT) {
            cudaError_t e = dmalloc_n(ctx, &w->HlcT, (size_t)ctx->Dc * ctx->n_l2);
            if (e != cudaSuccess) return diag_fail(ctx, HB_ERR_OOM, "Davidson transpose buffer");
        }
        w->HlcT_src = H->Hlc;
    }
    return HB_OK;
}

extern "C" int hb_diag(hb_ctx *ctx, const hb_blocks *H, int32_t k, double tol, int32_t max_iter, int32_t precond,
                       const double *v0, double *evals, double *evecs, hb_stats *st, void *stream) {
    if (!ctx || !H || !evals) return HB_ERR_INVALID_ARG;
    const int64_t n = ctx->dim;
    if (k < 1 || k > n || tol <= 0 || max_iter < 1) return diag_fail(ctx, HB_ERR_INVALID_ARG, "bad k, tol or max_iter");
    if ((ctx->Dc > 0 && !H->Hcc) || (ctx->Dc > 0 && ctx->n_l2 > 0 && !H->Hlc) ||
        (ctx->n_l2 > 0 && (!H->l2_row_ptr || !H->l2_col || !H->l2_val)))
        return diag_fail(ctx, HB_ERR_INVALID_ARG, "matrix blocks are NULL");
    const bool tensor = (precond & HB_DIAG_TENSOR) != 0;
    precond &= ~HB_DIAG_TENSOR;
    if (precond != HB_PRECOND_DIAG && precond != HB_PRECOND_MLP)
        return diag_fail(ctx, HB_ERR_INVALID_ARG, "precond must be HB_PRECOND_DIAG or HB_PRECOND_MLP (| HB_DIAG_TENSOR)");
    if (precond == HB_PRECOND_MLP && !ctx->mlp)
        return diag_fail(ctx, HB_ERR_INVALID_ARG, "HB_PRECOND_MLP without weights (hb_mlp_set)");
    cudaStream_t s = (cudaStream_t)stream;
    const int b = (int)std::min<int64_t>(n, k + std::max(4, std::min(16, k / 2)));
    const int mmax = (int)std::min<int64_t>(n, (int64_t)ctx->diag_basis * b);
    int rc = ensure_diag_work(ctx, H, mmax, s);
    if (rc != HB_OK) return rc;
    DiagWork *w = (DiagWork *)ctx->diag;
    Ops ops{ctx, H, s, n, ctx->Dc, ctx->n_l2, w};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    float ms_mv = 0.0f;
    if (ctx->Dc > 0 && ctx->n_l2 > 0) {
        dim3 g((unsigned)((ctx->Dc + 31) / 32), (unsigned)((ctx->n_l2 + 31) / 32));
        transpose_kernel<<<g, dim3(32, 8), 0, s>>>(H->Hlc, ctx->n_l2, ctx->Dc, w->HlcT);
        ++ops.launches;
    }
    if (tensor) {
        // slices of the fixed operands, once per call
        rc = setup_tensor_products(ctx, H, w, mmax, s);
        if (rc != HB_OK) return rc;
        ops.launches += 2;
    }
    diag_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(H->Hcc, ctx->Dc, H->l2_row_ptr, H->l2_col, H->l2_val,
                                                             ctx->n_l2, w->d);
    ++ops.launches;
    std::vector<double> dh(n);
    cudaMemcpyAsync(dh.data(), w->d, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    const int64_t ld = n;
    // --- initial block
    int m = 0;
    if (v0) {
        dim3 g((unsigned)((n + 255) / 256), k);
        import_kernel<<<g, 256, 0, s>>>(v0, k, n, w->V, ld);
        m = k;
    } else {
        std::vector<int32_t> ord(n);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return dh[a] < dh[c]; });
        const int q = b;
        cudaMemcpyAsync(w->idx, ord.data(), sizeof(int32_t) * q, cudaMemcpyHostToDevice, s);
        dim3 g((unsigned)((n + 255) / 256), q);
        unit_vectors_kernel<<<g, 256, 0, s>>>(w->V, ld, w->idx, q, n);
        m = q;
    }
    // orthonormalise the start block (SVQB) and take its products
    auto svqb = [&](double *blk, int q, int &kept) {
        std::vector<double> G, lam, U;
        ops.gram(blk, q, blk, q, ld, G);
        for (int a = 0; a < q; ++a)
            for (int c = 0; c < a; ++c) G[(size_t)a * q + c] = G[(size_t)c * q + a] = 0.5 * (G[(size_t)a * q + c] + G[(size_t)c * q + a]);
        // A block that is already nearly orthonormal (the second pass: every
        // |G - I| below 0.1, so cond(G) < 1.3) is finished by Cholesky,
        // G = L L^T and C = L^-T, whose orthogonality error is a few units of
        // rounding; the eigenvalues of such a G form one large cluster, which
        // the eigensolver would treat vector by vector.
        {
            double dev = 0.0;
            for (int a = 0; a < q; ++a)
                for (int c = 0; c < q; ++c) dev = std::max(dev, std::fabs(G[(size_t)a * q + c] - (a == c ? 1.0 : 0.0)));
            if (dev < 0.1) {
                std::vector<double> L(G);
                bool ok = true;
                for (int j = 0; j < q && ok; ++j) {
                    double d = L[(size_t)j * q + j];
                    for (int t2 = 0; t2 < j; ++t2) d -= L[(size_t)j * q + t2] * L[(size_t)j * q + t2];
                    if (!(d > 0.5)) { ok = false; break; }
                    const double ljj = std::sqrt(d);
                    L[(size_t)j * q + j] = ljj;
                    for (int i = j + 1; i < q; ++i) {
                        double v = L[(size_t)i * q + j];
                        for (int t2 = 0; t2 < j; ++t2) v -= L[(size_t)i * q + t2] * L[(size_t)j * q + t2];
                        L[(size_t)i * q + j] = v / ljj;
                    }
                }
                if (ok) {
                    // C = L^-T: upper triangular, column c solves L^T C[:, c] = e_c
                    std::vector<double> C((size_t)q * q, 0.0);
                    for (int c = 0; c < q; ++c)
                        for (int a = c; a >= 0; --a) {
                            double v = (a == c) ? 1.0 : 0.0;
                            for (int t2 = a + 1; t2 <= c; ++t2) v -= L[(size_t)t2 * q + a] * C[(size_t)t2 * q + c];
                            C[(size_t)a * q + c] = v / L[(size_t)a * q + a];
                        }
                    kept = q;
                    ops.combine(blk, q, C, q, w->X, ld, 0.0);
                    cudaMemcpyAsync(blk, w->X, sizeof(double) * (size_t)q * ld, cudaMemcpyDeviceToDevice, s);
                    return;
                }
            }
        }
        ops.eigh(q, G, lam, U, q);
        const double lmax = lam.empty() ? 0.0 : lam.back();
        std::vector<int> keep;
        for (int a = 0; a < q; ++a)
            if (lam[a] > 1e-14 * lmax && lam[a] > 1e-30) keep.push_back(a);
        kept = (int)keep.size();
        std::vector<double> C((size_t)q * std::max(kept, 1));
        for (int a = 0; a < q; ++a)
            for (int c = 0; c < kept; ++c) C[(size_t)a * kept + c] = U[(size_t)a * q + keep[c]] / std::sqrt(lam[keep[c]]);
        if (kept > 0) {
            ops.combine(blk, q, C, kept, w->X, ld, 0.0);
            cudaMemcpyAsync(blk, w->X, sizeof(double) * (size_t)kept * ld, cudaMemcpyDeviceToDevice, s);
        }
    };
    {
        int kept = 0;
        svqb(w->V, m, kept);
        m = kept;
    }
    ops.matvec(w->V, w->AV, m, ld);
    int iter = 0;
    bool converged = false;
    double maxres = 0.0;
    std::vector<double> theta;
    float *wts = nullptr;
    int fallbacks = 0;
    const int kStall = ctx->stall_iters;
    constexpr int kTcStall = 10;
    const double stall_fall = std::ldexp(1.0, -ctx->stall_log2);
    int refreshes = 0, fp64_iters = 0;
    std::vector<double> res_hist;
    // projected matrix T = V^T A V, kept up to date on the host: the full
    // product for the start block, one border V^T (A V_new) per iteration, and
    // diag(theta) for the Ritz vectors kept at a restart
    std::vector<double> Tp;
    ops.gram(w->V, m, w->AV, m, ld, Tp);
    for (iter = 1; iter <= max_iter; ++iter) {
        if (ops.force_fp64) ++fp64_iters;
        // Rayleigh-Ritz
        std::vector<double> T(Tp), S;
        for (int a = 0; a < m; ++a)
            for (int c = 0; c < a; ++c) T[(size_t)a * m + c] = T[(size_t)c * m + a] = 0.5 * (T[(size_t)a * m + c] + T[(size_t)c * m + a]);
        // Ritz vectors needed: b, and 2b when this iteration may restart
        const int nv = std::min(m, m + b > mmax ? 2 * b : b);
        ops.eigh(m, T, theta, S, nv);
        const int nr = std::min(m, b);
        std::vector<double> Sk((size_t)m * nr);
        for (int a = 0; a < m; ++a)
            for (int c = 0; c < nr; ++c) Sk[(size_t)a * nr + c] = S[(size_t)a * nv + c];
        ops.combine(w->V, m, Sk, nr, w->X, ld, 0.0);
        ops.combine(w->AV, m, Sk, nr, w->AX, ld, 0.0);
        // residuals (kept in AX) and their norms
        cudaMemcpyAsync(w->theta, theta.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, s);
        {
            dim3 g((unsigned)((n + 255) / 256), nr);
            residual_kernel<<<g, 256, 0, s>>>(w->AX, w->X, ld, w->theta, nr, n, w->AX);
            ++ops.launches;
        }
        std::vector<double> RR;
        ops.norms2(w->AX, nr, ld, RR);
        std::vector<int32_t> which;
        maxres = 0.0;
        for (int j = 0; j < nr; ++j) {
            const double r = std::sqrt(std::max(0.0, RR[(size_t)j]));
            if (j < k) maxres = std::max(maxres, r);
            if (r > tol) which.push_back(j);
        }
        bool done = true;
        for (int j = 0; j < k; ++j)
            if (std::sqrt(std::max(0.0, RR[(size_t)j])) > tol) done = false;
        // With tensor-core products the residuals carry a floor of their own:
        // the product errors E give the Ritz residual a component inside the
        // basis, (V^T E - sym(V^T E)) s, that no correction (orthogonal to
        // the basis) removes, and it grows with the basis.  When the largest
        // wanted residual, already within 1e4 tol, has not halved over
        // kTcStall iterations, the solve goes on from fresh FP64 products, as
        // after a converged check.
        const bool tc_stalled = w->tc && !ops.force_fp64 && (int)res_hist.size() >= kTcStall &&
                                maxres <= 1e4 * tol && maxres > 0.5 * res_hist[res_hist.size() - kTcStall];
        if (done || tc_stalled) {
            // The residuals above come from products carried through the
            // restarts (A X = (A V) S): the Rayleigh-Ritz step fits the errors
            // of those products, so they measure the residual of a perturbed
            // operator.  Confirm them with fresh FP64 products H X of the Ritz
            // vectors (the split-bf16 products err by about 2^-42 of each row
            // and vector scale, which for long delocalised vectors reaches
            // 1e-8 in norm).  The basis restarts from those vectors and
            // products; a solve that is not yet converged finishes with FP64
            // products (iterative refinement of the tensor-core solve).
            ops.force_fp64 = true;
            cudaMemcpyAsync(w->V, w->X, sizeof(double) * (size_t)nr * ld, cudaMemcpyDeviceToDevice, s);
            ops.matvec(w->V, w->AV, nr, ld);
            m = nr;
            ops.gram(w->V, m, w->AV, m, ld, Tp);
            cudaMemcpyAsync(w->AX, w->AV, sizeof(double) * (size_t)nr * ld, cudaMemcpyDeviceToDevice, s);
            {
                dim3 g((unsigned)((n + 255) / 256), nr);
                residual_kernel<<<g, 256, 0, s>>>(w->AX, w->X, ld, w->theta, nr, n, w->AX);
                ++ops.launches;
            }
            ops.norms2(w->AX, nr, ld, RR);
            which.clear();
            maxres = 0.0;
            for (int j = 0; j < nr; ++j) {
                const double r = std::sqrt(std::max(0.0, RR[(size_t)j]));
                if (j < k) maxres = std::max(maxres, r);
                if (r > tol) which.push_back(j);
            }
            done = true;
            for (int j = 0; j < k; ++j)
                if (std::sqrt(std::max(0.0, RR[(size_t)j])) > tol) done = false;
            ++refreshes;
            if (done) { converged = true; break; }
        }
        if (iter == max_iter) break;
        // corrections for the unconverged Ritz pairs (lowest first, at most b)
        if ((int)which.size() > b) which.resize(b);
        int q = (int)which.size();
        // thick restart when the basis would overflow: keep the 2b lowest Ritz
        // vectors (the residuals of the first nr stay in AX)
        if (m + q > mmax) {
            const int keep = std::min(m, std::min(2 * b, mmax - q));
            std::vector<double> Sr((size_t)m * keep);
            for (int a2 = 0; a2 < m; ++a2)
                for (int c = 0; c < keep; ++c) Sr[(size_t)a2 * keep + c] = S[(size_t)a2 * nv + c];
            ops.combine(w->V, m, Sr, keep, w->W2, ld, 0.0);
            cudaMemcpyAsync(w->V, w->W2, sizeof(double) * (size_t)keep * ld, cudaMemcpyDeviceToDevice, s);
            ops.combine(w->AV, m, Sr, keep, w->W2, ld, 0.0);
            cudaMemcpyAsync(w->AV, w->W2, sizeof(double) * (size_t)keep * ld, cudaMemcpyDeviceToDevice, s);
            m = keep;
            Tp.assign((size_t)m * m, 0.0);
            for (int a2 = 0; a2 < m; ++a2) Tp[(size_t)a2 * m + a2] = theta[a2];
        }
        if (m + q > mmax) q = mmax - m;
        if (q <= 0) break;
        cudaMemcpyAsync(w->idx, which.data(), sizeof(int32_t) * q, cudaMemcpyHostToDevice, s);
        // the learned factor is dropped for the rest of the solve when the
        // largest wanted residual has not fallen by 2^stall_log2 (halved by
        // default) over the last kStall iterations
        res_hist.push_back(maxres);
        if (precond == HB_PRECOND_MLP && (int)res_hist.size() > kStall &&
            maxres > stall_fall * res_hist[res_hist.size() - 1 - kStall]) {
            precond = HB_PRECOND_DIAG;
            wts = nullptr;
            ++fallbacks;
        }
        if (precond == HB_PRECOND_MLP) {
            int frc = mlp_weights_for(ctx, w, theta.data(), nr, &wts, s);
            if (frc != HB_OK) { wts = nullptr; ++fallbacks; }
        }
        double *Tn = w->V + (int64_t)m * ld;
        {
            dim3 g((unsigned)((n + 255) / 256), q);
            precond_kernel<<<g, 256, 0, s>>>(w->AX, ld, w->d, w->theta, w->idx, q, n, wts, Tn, ld);
            ++ops.launches;
        }
        // orthogonalise against the basis twice, then within the block
        for (int pass = 0; pass < 2; ++pass) ops.project_out(w->V, m, Tn, q, ld);
        int kept = 0;
        svqb(Tn, q, kept);
        if (kept == 0) break;
        {
            ops.project_out(w->V, m, Tn, kept, ld);
            int k2 = 0;
            svqb(Tn, kept, k2);
            kept = k2;
        }
        if (kept == 0) break;
        cudaEvent_t m0, m1;
        cudaEventCreate(&m0);
        cudaEventCreate(&m1);
        cudaEventRecord(m0, s);
        ops.matvec(Tn, w->AV + (int64_t)m * ld, kept, ld);
        cudaEventRecord(m1, s);
        cudaEventSynchronize(m1);
        float t = 0.0f;
        cudaEventElapsedTime(&t, m0, m1);
        ms_mv += t;
        cudaEventDestroy(m0);
        cudaEventDestroy(m1);
        {
            // border of T: rows 0 .. m+kept of V against the new products
            std::vector<double> G;
            const int mn = m + kept;
            ops.gram(w->V, mn, w->AV + (int64_t)m * ld, kept, ld, G);
            std::vector<double> Tn2((size_t)mn * mn, 0.0);
            for (int a2 = 0; a2 < m; ++a2)
                for (int c = 0; c < m; ++c) Tn2[(size_t)a2 * mn + c] = Tp[(size_t)a2 * m + c];
            for (int a2 = 0; a2 < mn; ++a2)
                for (int c = 0; c < kept; ++c) {
                    Tn2[(size_t)a2 * mn + m + c] = G[(size_t)a2 * kept + c];
                    if (a2 < m) Tn2[(size_t)(m + c) * mn + a2] = G[(size_t)a2 * kept + c];
                }
            Tp.swap(Tn2);
        }
        m += kept;
    }
    for (int j = 0; j < k && j < (int)theta.size(); ++j) evals[j] = theta[j];
    if (evecs) {
        dim3 g((unsigned)((n + 255) / 256), k);
        export_kernel<<<g, 256, 0, s>>>(w->X, ld, k, n, evecs);
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return diag_fail(ctx, HB_ERR_CUDA, std::string("Davidson: ") + cudaGetErrorString(e));
    if (w->tc) {
        int word = 0;
        cudaMemcpy(&word, w->err, sizeof(int), cudaMemcpyDeviceToHost);
        release_tensor_products(ctx, w);
        if (word) return diag_fail(ctx, HB_ERR_TIMEOUT, "Davidson tensor-core product gave up waiting");
    }
    if (st) {
        memset(st, 0, sizeof(*st));
        st->ms_total = ms;
        st->iterations = std::min(iter, max_iter);
        st->max_residual = maxres;
        st->ms_matvec = ms_mv;
        st->ms_rr = (float)ops.ms_eigh;
        st->ms_gram = (float)ops.ms_gram;
        st->ms_combine = (float)ops.ms_combine;
        st->fp64_iterations = fp64_iters;
        st->kernel_launches = ops.launches;
        st->mlp_fallbacks = fallbacks;
        st->proj_gflop = (int32_t)std::min(2.0e9, ops.proj_flops / 1e9 + 0.5);
    }
    if (!converged) return diag_fail(ctx, HB_ERR_NOT_CONVERGED, "Davidson did not converge in max_iter iterations");
    return HB_OK;
}

void hb::release_diag(hb_ctx *ctx) {
    DiagWork *w = (DiagWork *)ctx->diag;
    if (!w) return;
    release_tensor_products(ctx, w);
    for (void *p : {(void *)w->V, (void *)w->AV, (void *)w->X, (void *)w->AX, (void *)w->W2, (void *)w->d, (void *)w->partial,
                    (void *)w->small, (void *)w->proj, (void *)w->theta, (void *)w->idx, (void *)w->HlcT,
                    (void *)w->XT})
        dfree(ctx, p);
    delete w;
    ctx->diag = nullptr;
}
