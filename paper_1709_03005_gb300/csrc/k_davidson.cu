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
#include <cmath>
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

// Y[j][l] += sum_p val[p] X[j][col[p]] over CSR rows l; one warp per row, lanes
// over vectors (in groups of 32), entries in order.
__global__ void spmm_csr_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                const double *__restrict__ val, int rows, const double *__restrict__ X, int64_t ldx,
                                int q, double *__restrict__ Y, int64_t ldy) {
    const int lane = threadIdx.x & 31;
    const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (l >= rows) return;
    const int64_t b = rp[l], e = rp[l + 1];
    for (int j0 = 0; j0 < q; j0 += 32) {
        const int j = j0 + lane;
        if (j >= q) break;
        double acc = 0.0;
        for (int64_t p = b; p < e; ++p) acc = fma(__ldg(val + p), __ldg(X + (int64_t)j * ldx + __ldg(col + p)), acc);
        Y[(int64_t)j * ldy + l] += acc;
    }
}

// partial[c][a][b] = sum_{i in chunk c} X[a][i] Y[b][i]
constexpr int kGramChunk = 2048;
__global__ void gram_partial_kernel(const double *__restrict__ X, int64_t ldx, int p, const double *__restrict__ Y,
                                    int64_t ldy, int q, int64_t n, double *__restrict__ partial) {
    const int c = blockIdx.x;
    const int64_t i0 = (int64_t)c * kGramChunk, i1 = (n < i0 + kGramChunk) ? n : i0 + kGramChunk;
    for (int t = threadIdx.x + blockIdx.y * blockDim.x; t < p * q; t += blockDim.x * gridDim.y) {
        const int a = t / q, b = t % q;
        const double *x = X + (int64_t)a * ldx, *y = Y + (int64_t)b * ldy;
        double acc = 0.0;
        for (int64_t i = i0; i < i1; ++i) acc = fma(x[i], y[i], acc);
        partial[(int64_t)c * p * q + t] = acc;
    }
}

__global__ void reduce_kernel(const double *__restrict__ partial, int chunks, int nout, double *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nout) return;
    double acc = 0.0;
    for (int c = 0; c < chunks; ++c) acc += partial[(int64_t)c * nout + t];
    out[t] = acc;
}

// Y[j][i] = beta * Y[j][i] + sum_a C[a][j] X[a][i]   (a < p, j < q), C on device [p][q]
__global__ void combine_kernel(const double *__restrict__ X, int64_t ldx, int p, const double *__restrict__ C, int q,
                               int64_t n, double *__restrict__ Y, int64_t ldy, double beta) {
    extern __shared__ double cs[];   // [p][16]
    const int j0 = blockIdx.y * 16;
    const int nq = min(16, q - j0);
    for (int t = threadIdx.x; t < p * 16; t += blockDim.x) {
        const int a = t / 16, jj = t % 16;
        cs[t] = jj < nq ? C[(int64_t)a * q + j0 + jj] : 0.0;
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc[16];
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) acc[jj] = 0.0;
    for (int a = 0; a < p; ++a) {
        const double x = __ldg(X + (int64_t)a * ldx + i);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) acc[jj] = fma(cs[a * 16 + jj], x, acc[jj]);
    }
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
void hb::small_eigh(int n, std::vector<double> A, std::vector<double> &w, std::vector<double> &V) {
    w.assign(n, 0.0);
    V.assign((size_t)n * n, 0.0);
    if (n == 0) return;
    if (n == 1) { w[0] = A[0]; V[0] = 1.0; return; }
    // z holds the accumulated orthogonal transformation, row-major z[i][j]
    std::vector<double> z(A), d(n), e(n);
    auto Z = [&](int i, int j) -> double & { return z[(size_t)i * n + j]; };
    // --- Householder tridiagonalisation (rows from the bottom up)
    for (int i = n - 1; i > 0; --i) {
        const int l = i - 1;
        double h = 0.0, scale = 0.0;
        if (l > 0) {
            for (int k = 0; k <= l; ++k) scale += std::fabs(Z(i, k));
            if (scale == 0.0) {
                e[i] = Z(i, l);
            } else {
                for (int k = 0; k <= l; ++k) { Z(i, k) /= scale; h += Z(i, k) * Z(i, k); }
                double f = Z(i, l);
                double g = f >= 0.0 ? -std::sqrt(h) : std::sqrt(h);
                e[i] = scale * g;
                h -= f * g;
                Z(i, l) = f - g;
                f = 0.0;
                for (int j = 0; j <= l; ++j) {
                    Z(j, i) = Z(i, j) / h;
                    g = 0.0;
                    for (int k = 0; k <= j; ++k) g += Z(j, k) * Z(i, k);
                    for (int k = j + 1; k <= l; ++k) g += Z(k, j) * Z(i, k);
                    e[j] = g / h;
                    f += e[j] * Z(i, j);
                }
                const double hh = f / (h + h);
                for (int j = 0; j <= l; ++j) {
                    f = Z(i, j);
                    e[j] = g = e[j] - hh * f;
                    for (int k = 0; k <= j; ++k) Z(j, k) -= (f * e[k] + g * Z(i, k));
                }
            }
        } else {
            e[i] = Z(i, l);
        }
        d[i] = h;
    }
    d[0] = 0.0;
    e[0] = 0.0;
    for (int i = 0; i < n; ++i) {
        const int l = i - 1;
        if (d[i] != 0.0) {
            for (int j = 0; j <= l; ++j) {
                double g = 0.0;
                for (int k = 0; k <= l; ++k) g += Z(i, k) * Z(k, j);
                for (int k = 0; k <= l; ++k) Z(k, j) -= g * Z(k, i);
            }
        }
        d[i] = Z(i, i);
        Z(i, i) = 1.0;
        for (int j = 0; j <= l; ++j) Z(j, i) = Z(i, j) = 0.0;
    }
    // --- implicit QL on (d, e) with accumulation into z
    for (int i = 1; i < n; ++i) e[i - 1] = e[i];
    e[n - 1] = 0.0;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        int m;
        do {
            for (m = l; m < n - 1; ++m) {
                const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
                if (std::fabs(e[m]) <= 1e-16 * dd) break;
            }
            if (m != l) {
                if (++iter > 60) break;
                double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
                double r = std::hypot(g, 1.0);
                g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? std::fabs(r) : -std::fabs(r)));
                double s = 1.0, c = 1.0, p = 0.0;
                int i;
                for (i = m - 1; i >= l; --i) {
                    double f = s * e[i], b = c * e[i];
                    e[i + 1] = (r = std::hypot(f, g));
                    if (r == 0.0) {
                        d[i + 1] -= p;
                        e[m] = 0.0;
                        break;
                    }
                    s = f / r;
                    c = g / r;
                    g = d[i + 1] - p;
                    r = (d[i] - g) * s + 2.0 * c * b;
                    d[i + 1] = g + (p = s * r);
                    g = c * r - b;
                    for (int k = 0; k < n; ++k) {
                        f = Z(k, i + 1);
                        Z(k, i + 1) = s * Z(k, i) + c * f;
                        Z(k, i) = c * Z(k, i) - s * f;
                    }
                }
                if (r == 0.0 && i >= l) continue;
                d[l] -= p;
                e[l] = g;
                e[m] = 0.0;
            }
        } while (m != l);
    }
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return d[a] < d[b]; });
    for (int j = 0; j < n; ++j) {
        w[j] = d[ord[j]];
        for (int i = 0; i < n; ++i) V[(size_t)i * n + j] = Z(i, ord[j]);
    }
}

extern "C" int hb_test_symeig(int n, const double *A, double *w, double *V) {
    std::vector<double> a(A, A + (size_t)n * n), ww, vv;
    hb::small_eigh(n, a, ww, vv);
    std::memcpy(w, ww.data(), sizeof(double) * n);
    std::memcpy(V, vv.data(), sizeof(double) * (size_t)n * n);
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
    int launches = 0;

    // Y[0:q] = H X[0:q], vectors stored as rows of length ld
    void matvec(const double *X, double *Y, int q, int64_t ld) {
        if (q <= 0) return;
        if (w->tc) {
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
                spmm_csr_kernel<<<(unsigned)((nl + 7) / 8), 256, 0, s>>>(H->l2_row_ptr, H->l2_col, H->l2_val, (int)nl,
                                                                         X + Dc, ld, q, Y + Dc, ld);
                ++launches;
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
            spmm_csr_kernel<<<(unsigned)((nl + 7) / 8), 256, 0, s>>>(H->l2_row_ptr, H->l2_col, H->l2_val, (int)nl,
                                                                     X + Dc, ld, q, Y + Dc, ld);
            ++launches;
        }
    }

    // G[a][b] = X[a] . Y[b] on the host (p x q)
    void gram(const double *X, int p, const double *Y, int q, int64_t ld, std::vector<double> &G) {
        const int chunks = (int)((n + kGramChunk - 1) / kGramChunk);
        dim3 g(chunks, std::max(1, std::min(8, (p * q + 255) / 256)));
        gram_partial_kernel<<<g, 256, 0, s>>>(X, ld, p, Y, ld, q, n, w->partial);
        reduce_kernel<<<(p * q + 255) / 256, 256, 0, s>>>(w->partial, chunks, p * q, w->small);
        launches += 2;
        G.resize((size_t)p * q);
        cudaMemcpyAsync(G.data(), w->small, sizeof(double) * p * q, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
    }

    // Y[0:q] = beta Y + X[0:p]^T C, C host [p][q]
    void combine(const double *X, int p, const std::vector<double> &C, int q, double *Y, int64_t ld, double beta) {
        cudaMemcpyAsync(w->small, C.data(), sizeof(double) * p * q, cudaMemcpyHostToDevice, s);
        dim3 g((unsigned)((n + 255) / 256), (q + 15) / 16);
        combine_kernel<<<g, 256, sizeof(double) * p * 16, s>>>(X, ld, p, w->small, q, n, Y, ld, beta);
        ++launches;
        cudaStreamSynchronize(s);   // w->small is reused by the next call
    }
};

}  // namespace

static int diag_fail(hb_ctx *ctx, int code, const std::string &m) {
    ctx->err = m;
    return code;
}

static void release_tensor_products(DiagWork *w) {
    dense_operand_free(&w->A1);
    dense_operand_free(&w->A2);
    dense_operand_free(&w->Xs);
    if (w->part) cudaFree(w->part);
    if (w->err) cudaFree(w->err);
    w->part = nullptr;
    w->err = nullptr;
    w->tc = false;
}

// Slices of [Hcc | Hlc^T] and of Hlc (fixed during the solve), the vector
// slice buffer for up to mmax vectors and the split-K scratch.
static int setup_tensor_products(hb_ctx *ctx, const hb_blocks *H, DiagWork *w, int mmax, cudaStream_t s) {
    release_tensor_products(w);
    const int64_t n = ctx->dim, Dc = ctx->Dc, nl = ctx->n_l2;
    const int S = ctx->split_slices >= 2 && ctx->split_slices <= 6 ? ctx->split_slices : 6;
    w->S = S;
    std::string err;
    const int K1 = (int)((n + 63) / 64 * 64), K2 = (int)((Dc + 63) / 64 * 64);
    int rc = dense_operand_alloc(S, mmax, K1, &w->Xs, &err);
    if (rc == HB_OK && Dc > 0) rc = dense_operand_alloc(S, Dc, K1, &w->A1, &err);
    if (rc == HB_OK && Dc > 0 && nl > 0) rc = dense_operand_alloc(S, nl, K2, &w->A2, &err);
    size_t part = 1;
    int per = 0;
    if (Dc > 0) part = std::max(part, (size_t)dense_splits(Dc, 1, K1 / 64, &per) * mmax * Dc);
    if (Dc > 0 && nl > 0) part = std::max(part, (size_t)dense_splits(nl, 1, K2 / 64, &per) * mmax * nl);
    cudaError_t e = cudaSuccess;
    if (rc == HB_OK) e = cudaMalloc(&w->part, sizeof(float2) * part);
    if (rc == HB_OK && e == cudaSuccess) e = cudaMalloc(&w->err, sizeof(int));
    if (rc == HB_OK && e == cudaSuccess) e = cudaMemsetAsync(w->err, 0, sizeof(int), s);
    if (rc == HB_OK && e != cudaSuccess) {
        rc = HB_ERR_OOM;
        err = std::string("Davidson tensor-core scratch: ") + cudaGetErrorString(e);
    }
    if (rc != HB_OK) {
        release_tensor_products(w);
        return diag_fail(ctx, rc, err);
    }
    if (Dc > 0) dense_operand_fill(w->A1, S, H->Hcc, Dc, (int)Dc, nl > 0 ? w->HlcT : nullptr, nl, (int)nl, Dc, s);
    if (Dc > 0 && nl > 0) dense_operand_fill(w->A2, S, H->Hlc, Dc, (int)Dc, nullptr, 0, 0, nl, s);
    w->tc = true;
    return HB_OK;
}

int hb::ensure_diag_work(hb_ctx *ctx, const hb_blocks *H, int mmax, cudaStream_t s) {
    DiagWork *w = (DiagWork *)ctx->diag;
    const int64_t n = ctx->dim;
    if (!w) {
        w = new DiagWork();
        ctx->diag = w;
    }
    if (w->mmax < mmax || w->n != n) {
        auto fr = [](void *p) { if (p) cudaFree(p); };
        fr(w->V); fr(w->AV); fr(w->X); fr(w->AX); fr(w->W2); fr(w->d); fr(w->partial); fr(w->small); fr(w->theta);
        fr(w->idx);
        w->V = w->AV = w->X = w->AX = w->W2 = w->d = w->partial = w->small = w->theta = nullptr;
        w->idx = nullptr;
        const size_t vec = sizeof(double) * (size_t)mmax * n;
        cudaError_t e = cudaMalloc(&w->V, vec);
        if (e == cudaSuccess) e = cudaMalloc(&w->AV, vec);
        if (e == cudaSuccess) e = cudaMalloc(&w->X, vec);
        if (e == cudaSuccess) e = cudaMalloc(&w->AX, vec);
        if (e == cudaSuccess) e = cudaMalloc(&w->W2, vec);
        if (e == cudaSuccess) e = cudaMalloc(&w->d, sizeof(double) * n);
        const int chunks = (int)((n + kGramChunk - 1) / kGramChunk);
        if (e == cudaSuccess) e = cudaMalloc(&w->partial, sizeof(double) * (size_t)chunks * mmax * mmax);
        if (e == cudaSuccess) e = cudaMalloc(&w->small, sizeof(double) * (size_t)mmax * mmax);
        if (e == cudaSuccess) e = cudaMalloc(&w->theta, sizeof(double) * mmax);
        if (e == cudaSuccess) e = cudaMalloc(&w->idx, sizeof(int32_t) * mmax);
        if (e != cudaSuccess) return diag_fail(ctx, HB_ERR_OOM, std::string("Davidson workspace: ") + cudaGetErrorString(e));
        w->mmax = mmax;
        w->n = n;
    }
    if (ctx->Dc > 0 && ctx->n_l2 > 0 && (!w->HlcT || w->HlcT_src != H->Hlc)) {
        if (!w->HlcT) {
            cudaError_t e = cudaMalloc(&w->HlcT, sizeof(double) * (size_t)ctx->Dc * ctx->n_l2);
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
    const int mmax = (int)std::min<int64_t>(n, std::max(5 * b, k + 4 * b));
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
        small_eigh(q, G, lam, U);
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
    for (iter = 1; iter <= max_iter; ++iter) {
        // Rayleigh-Ritz
        std::vector<double> T, S;
        ops.gram(w->V, m, w->AV, m, ld, T);
        for (int a = 0; a < m; ++a)
            for (int c = 0; c < a; ++c) T[(size_t)a * m + c] = T[(size_t)c * m + a] = 0.5 * (T[(size_t)a * m + c] + T[(size_t)c * m + a]);
        small_eigh(m, T, theta, S);
        const int nr = std::min(m, b);
        std::vector<double> Sk((size_t)m * nr);
        for (int a = 0; a < m; ++a)
            for (int c = 0; c < nr; ++c) Sk[(size_t)a * nr + c] = S[(size_t)a * m + c];
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
        ops.gram(w->AX, nr, w->AX, nr, ld, RR);
        std::vector<int32_t> which;
        maxres = 0.0;
        for (int j = 0; j < nr; ++j) {
            const double r = std::sqrt(std::max(0.0, RR[(size_t)j * nr + j]));
            if (j < k) maxres = std::max(maxres, r);
            if (r > tol) which.push_back(j);
        }
        bool done = true;
        for (int j = 0; j < k; ++j)
            if (std::sqrt(std::max(0.0, RR[(size_t)j * nr + j])) > tol) done = false;
        if (done) { converged = true; break; }
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
                for (int c = 0; c < keep; ++c) Sr[(size_t)a2 * keep + c] = S[(size_t)a2 * m + c];
            ops.combine(w->V, m, Sr, keep, w->W2, ld, 0.0);
            cudaMemcpyAsync(w->V, w->W2, sizeof(double) * (size_t)keep * ld, cudaMemcpyDeviceToDevice, s);
            ops.combine(w->AV, m, Sr, keep, w->W2, ld, 0.0);
            cudaMemcpyAsync(w->AV, w->W2, sizeof(double) * (size_t)keep * ld, cudaMemcpyDeviceToDevice, s);
            m = keep;
        }
        if (m + q > mmax) q = mmax - m;
        if (q <= 0) break;
        cudaMemcpyAsync(w->idx, which.data(), sizeof(int32_t) * q, cudaMemcpyHostToDevice, s);
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
        for (int pass = 0; pass < 2; ++pass) {
            std::vector<double> C;
            ops.gram(w->V, m, Tn, q, ld, C);
            for (double &x : C) x = -x;
            ops.combine(w->V, m, C, q, Tn, ld, 1.0);
        }
        int kept = 0;
        svqb(Tn, q, kept);
        if (kept == 0) break;
        for (int pass = 0; pass < 1; ++pass) {
            std::vector<double> C;
            ops.gram(w->V, m, Tn, kept, ld, C);
            for (double &x : C) x = -x;
            ops.combine(w->V, m, C, kept, Tn, ld, 1.0);
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
        release_tensor_products(w);
        if (word) return diag_fail(ctx, HB_ERR_TIMEOUT, "Davidson tensor-core product gave up waiting");
    }
    if (st) {
        memset(st, 0, sizeof(*st));
        st->ms_total = ms;
        st->iterations = std::min(iter, max_iter);
        st->max_residual = maxres;
        st->ms_matvec = ms_mv;
        st->kernel_launches = ops.launches;
        st->mlp_fallbacks = fallbacks;
    }
    if (!converged) return diag_fail(ctx, HB_ERR_NOT_CONVERGED, "Davidson did not converge in max_iter iterations");
    return HB_OK;
}

void hb::release_diag(hb_ctx *ctx) {
    DiagWork *w = (DiagWork *)ctx->diag;
    if (!w) return;
    release_tensor_products(w);
    for (void *p : {(void *)w->V, (void *)w->AV, (void *)w->X, (void *)w->AX, (void *)w->W2, (void *)w->d, (void *)w->partial,
                    (void *)w->small, (void *)w->theta, (void *)w->idx, (void *)w->HlcT})
        if (p) cudaFree(p);
    delete w;
    ctx->diag = nullptr;
}
