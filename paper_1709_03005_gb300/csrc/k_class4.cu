// K4: class 4, continuum x L2 (Eq. 5).
//
// For L2 function l and target group g:
//   H~[l][(g n j)] = sum_{m partners of l} c_mn <D_m + j|H|chi_l>
// The classified (m, l) pairs (D_m within a single substitution of chi_l, so
// the (N+1)-electron pair is within a double excitation) are the prototypes;
// each gives, for every continuum orbital j, one or two integrals of the form
// (ab|c j) (plus h_jt for a single excitation), all contiguous in j in the
// (tt|tc) class array, so the threads of a block read them coalesced.
// A block owns one L2 row and a tile of continuum orbitals (one per thread)
// and keeps a tile of target states in registers; the CI rows of a batch of
// partners are staged in shared memory.
//   plain build: prototype values and the rank-1 accumulation in FP64;
//   mixed build: everything in double-float on the FP32 pipes (the FP64 pipe
//   of this part is 64 times narrower): the integrals, h and the CI vectors are
//   kept as (hi, lo) float pairs, the prototype sums use double-float adds,
//   the products c * y are exact by FMA and the accumulation is TwoSum based
//   (about 44 significant bits); the state tile and the thread count follow
//   the group's state and continuum counts.
#include "hb_df.cuh"
#include "hb_tasks.cuh"

namespace hb {

namespace {

constexpr int kJ = 128;
constexpr int kNS = 32;
constexpr int kBatch = 32;

__device__ __forceinline__ double x4(const Ints &I, int a, int b, int c, int j) {
    // (a b | c j), target a, b, c and continuum index j
    return __ldg(I.tttc + pair_idx(a, b) * ((int64_t)I.n_to * I.n_co) + (int64_t)c * I.n_co + j);
}

template <int W>
__device__ double prototype_value(const Ints &I, const hb_pair &r, const uint64_t *__restrict__ D, int j,
                                  int cont_spin) {
    const int sb = 64 * W;
    if (r.degree == 1) {
        // chi = D + t (spin cont_spin): single excitation t -> j
        const int t = r.hole[0] % sb;
        double v = __ldg(I.h + (int64_t)(I.n_to + j) * I.n_orb + t);
#pragma unroll
        for (int w = 0; w < 2 * W; ++w) {
            uint64_t x = __ldg(D + w);
            const int s = w / W;
            while (x) {
                const int k = 64 * (w % W) + __ffsll((long long)x) - 1;
                x &= x - 1;
                v += x4(I, k, k, t, j);                    // (jt|kk)
                if (s == cont_spin) v -= x4(I, k, t, k, j); // (jk|kt)
            }
        }
        return r.phase * v;
    }
    // degree 2: holes h1 < h2 in chi, particles {q, continuum} in D + j
    const int h1 = r.hole[0], h2 = r.hole[1], q = r.part[0];
    const int kq = 2 * q, kv = cont_spin == 0 ? 2 * 64 * W - 1 : 2 * 128 * W - 1;
    const int s1 = h1 / sb, s2 = h2 / sb, sq = q / sb;
    const int o1 = h1 % sb, o2 = h2 % sb, oq = q % sb;
    double dir = 0.0, exc = 0.0;
    if (kq < kv) {
        // p1 = q, p2 = continuum
        if (sq == s1 && cont_spin == s2) dir = x4(I, oq, o1, o2, j);   // (q h1|j h2)
        if (sq == s2 && cont_spin == s1) exc = x4(I, oq, o2, o1, j);   // (q h2|j h1)
    } else {
        // p1 = continuum, p2 = q
        if (cont_spin == s1 && sq == s2) dir = x4(I, oq, o2, o1, j);   // (j h1|q h2)
        if (cont_spin == s2 && sq == s1) exc = x4(I, oq, o1, o2, j);   // (j h2|q h1)
    }
    return r.phase * (dir - exc);
}

template <int W>
__global__ void __launch_bounds__(kJ)
class4_kernel(const C4Task *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    __shared__ double cs[kBatch][kNS];
    __shared__ hb_pair rs[kBatch];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const C4Task &T = tasks[ti];
    const Ints I = T.I;
    const hb_pair *__restrict__ pairs = T.pairs;
    const uint64_t *__restrict__ dets = T.dets;
    const double *__restrict__ C = T.C;
    const int ns = T.ns, cf = T.cf, cn = T.cn, cont_spin = T.cont_spin;
    const int lb = (int)(blockIdx.x - blk[ti]);
    const int l = lb / T.ny;
    const int jl = (lb % T.ny) * kJ + threadIdx.x;
    const bool jv = jl < cn;
    const int j = cf + (jv ? jl : 0);
    const int64_t b = T.row_ptr[l], e = T.row_ptr[l + 1];
    for (int n0 = 0; n0 < ns; n0 += kNS) {
        const int nc = min(kNS, ns - n0);
        double acc[kNS];
#pragma unroll
        for (int n = 0; n < kNS; ++n) acc[n] = 0.0;
        for (int64_t p0 = b; p0 < e; p0 += kBatch) {
            const int cnt = (int)(e - p0 < kBatch ? e - p0 : kBatch);
            __syncthreads();
            if (threadIdx.x < cnt) rs[threadIdx.x] = pairs[p0 + threadIdx.x];
            __syncthreads();
            for (int t = threadIdx.x; t < cnt * kNS; t += kJ) {
                const int i = t / kNS, n = t % kNS;
                cs[i][n] = n < nc ? C[(int64_t)rs[i].col * ns + n0 + n] : 0.0;
            }
            __syncthreads();
            for (int i = 0; i < cnt; ++i) {
                const hb_pair r = rs[i];
                const double y = prototype_value<W>(I, r, dets + (int64_t)r.col * 2 * W, j, cont_spin);
#pragma unroll
                for (int n = 0; n < kNS; ++n) acc[n] = fma(cs[i][n], y, acc[n]);
            }
        }
        if (jv) {
            double *out = T.Hlc + (int64_t)l * T.ld + T.col_off + jl;
#pragma unroll
            for (int n = 0; n < kNS; ++n)
                if (n < nc) out[(int64_t)(n0 + n) * cn] = acc[n];
        }
    }
}

// ------------------------------------------------------- double-float path
__device__ __forceinline__ float2 x4df(const C4Task &T, int a, int b, int c, int j) {
    return __ldg(T.tttc_df + pair_idx(a, b) * ((int64_t)T.I.n_to * T.I.n_co) + (int64_t)c * T.I.n_co + j);
}

template <int W>
__device__ __forceinline__ void prototype_df(const C4Task &T, const hb_pair &r, const uint64_t *__restrict__ D,
                                             int j, float &vh, float &vl) {
    const int sb = 64 * W;
    const int cont_spin = T.cont_spin;
    if (r.degree == 1) {
        // chi = D + t (spin cont_spin): single excitation t -> j
        const int t = r.hole[0] % sb;
        const float2 h = __ldg(T.h_df + (int64_t)(T.I.n_to + j) * T.I.n_orb + t);
        vh = h.x;
        vl = h.y;
#pragma unroll
        for (int w = 0; w < 2 * W; ++w) {
            uint64_t x = __ldg(D + w);
            const int s = w / W;
            while (x) {
                const int k = 64 * (w % W) + __ffsll((long long)x) - 1;
                x &= x - 1;
                const float2 a = x4df(T, k, k, t, j);                 // (jt|kk)
                df_add2(vh, vl, a.x, a.y);
                if (s == cont_spin) {
                    const float2 b = x4df(T, k, t, k, j);             // (jk|kt)
                    df_add2(vh, vl, -b.x, -b.y);
                }
            }
        }
    } else {
        // degree 2: holes h1 < h2 in chi, particles {q, continuum} in D + j
        const int h1 = r.hole[0], h2 = r.hole[1], q = r.part[0];
        const int kq = 2 * q, kv = cont_spin == 0 ? 2 * 64 * W - 1 : 2 * 128 * W - 1;
        const int s1 = h1 / sb, s2 = h2 / sb, sq = q / sb;
        const int o1 = h1 % sb, o2 = h2 % sb, oq = q % sb;
        float2 dir = make_float2(0.0f, 0.0f), exc = make_float2(0.0f, 0.0f);
        if (kq < kv) {
            if (sq == s1 && cont_spin == s2) dir = x4df(T, oq, o1, o2, j);   // (q h1|j h2)
            if (sq == s2 && cont_spin == s1) exc = x4df(T, oq, o2, o1, j);   // (q h2|j h1)
        } else {
            if (cont_spin == s1 && sq == s2) dir = x4df(T, oq, o2, o1, j);   // (j h1|q h2)
            if (cont_spin == s2 && sq == s1) exc = x4df(T, oq, o1, o2, j);   // (j h2|q h1)
        }
        vh = dir.x;
        vl = dir.y;
        df_add2(vh, vl, -exc.x, -exc.y);
    }
    if (r.phase < 0) {
        vh = -vh;
        vl = -vl;
    }
}

// Block = blockDim.x continuum orbitals (32, 64 or 128) of one L2 row; NS
// target states per pass.
template <int W, int NS>
__global__ void __launch_bounds__(kJ, NS <= 24 ? 6 : 1)
class4_df_kernel(const C4Task *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    __shared__ float2 cs[kBatch][NS];
    __shared__ hb_pair rs[kBatch];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const C4Task &T = tasks[ti];
    const int JT = blockDim.x;
    const int ns = T.ns, cn = T.cn;
    const int lb = (int)(blockIdx.x - blk[ti]);
    const int l = lb / T.ny;
    const int jl = (lb % T.ny) * JT + threadIdx.x;
    const bool jv = jl < cn;
    const int j = T.cf + (jv ? jl : 0);
    const int64_t b = T.row_ptr[l], e = T.row_ptr[l + 1];
    for (int n0 = 0; n0 < ns; n0 += NS) {
        const int nc = min(NS, ns - n0);
        float ahi[NS], alo[NS];
#pragma unroll
        for (int n = 0; n < NS; ++n) { ahi[n] = 0.0f; alo[n] = 0.0f; }
        for (int64_t p0 = b; p0 < e; p0 += kBatch) {
            const int cnt = (int)(e - p0 < kBatch ? e - p0 : kBatch);
            __syncthreads();
            for (int t = threadIdx.x; t < cnt; t += JT) rs[t] = T.pairs[p0 + t];
            __syncthreads();
            for (int t = threadIdx.x; t < cnt * NS; t += JT) {
                const int i = t / NS, n = t % NS;
                cs[i][n] = n < nc ? __ldg(T.C_df + (int64_t)rs[i].col * ns + n0 + n) : make_float2(0.0f, 0.0f);
            }
            __syncthreads();
            for (int i = 0; i < cnt; ++i) {
                const hb_pair r = rs[i];
                float yh, yl;
                prototype_df<W>(T, r, T.dets + (int64_t)r.col * 2 * W, j, yh, yl);
#pragma unroll
                for (int n = 0; n < NS; ++n) {
                    const float2 c = cs[i][n];
                    const float ph = c.x * yh;
                    const float pe = fmaf(c.x, yh, -ph);              // exact error of ph
                    const float pl = fmaf(c.x, yl, fmaf(c.y, yh, pe));
                    float sum, err;
                    df_two_sum(ahi[n], ph, sum, err);
                    ahi[n] = sum;
                    alo[n] = __fadd_rn(alo[n], __fadd_rn(err, pl));
                }
            }
            // renormalise once per batch so the low words stay small
#pragma unroll
            for (int n = 0; n < NS; ++n) {
                const float s = __fadd_rn(ahi[n], alo[n]);
                alo[n] = __fsub_rn(alo[n], __fsub_rn(s, ahi[n]));
                ahi[n] = s;
            }
        }
        if (jv) {
            double *out = T.Hlc + (int64_t)l * T.ld + T.col_off + jl;
#pragma unroll
            for (int n = 0; n < NS; ++n)
                if (n < nc) out[(int64_t)(n0 + n) * cn] = df_to_double(ahi[n], alo[n]);
        }
    }
}

__global__ void split_df_kernel(const double *__restrict__ x, int64_t n, float2 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    const float h = (float)v;
    out[i] = make_float2(h, (float)(v - (double)h));
}

}  // namespace

int class4_ny(int cn, int jt) { return (cn + jt - 1) / jt; }
int64_t blocks_class4(int n_l2, int cn, int jt) { return cn > 0 ? (int64_t)n_l2 * class4_ny(cn, jt) : 0; }

// State tile and thread count of the mixed kernel for a group (host side):
// the fewest passes over the states, then the smallest tile; the continuum
// tile that leaves the fewest idle threads (ties to the larger block).
void class4_shape(int ns, int cn, int *ns_tile, int *jt) {
    // passes of at most 32 states (larger tiles cost more in registers and
    // occupancy than the prototype values recomputed per pass), the state
    // tile rounded up to a multiple of 4 (8 beyond 32)
    const int passes = (ns + 31) / 32;
    const int need = (ns + passes - 1) / passes;
    *ns_tile = need <= 4 ? 4 : (need + 3) / 4 * 4;
    int best = 128;
    int64_t best_idle = (int64_t)((cn + 127) / 128) * 128 - cn;
    for (int t : {64, 32}) {
        const int64_t idle = (int64_t)((cn + t - 1) / t) * t - cn;
        if (idle < best_idle) { best = t; best_idle = idle; }
    }
    *jt = best;
}

void split_df(const double *x, int64_t n, float2 *out, cudaStream_t s) {
    if (n <= 0) return;
    split_df_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, out);
}

int g_class4(const Grouped<C4Task> &g, int W, int dfloat, int ns_tile, int jt, cudaStream_t s) {
    if (g.blocks <= 0) return 0;
    const unsigned grid = (unsigned)g.blocks;
    if (!dfloat) {
        switch (W) {
            case 1: class4_kernel<1><<<grid, kJ, 0, s>>>(g.tasks, g.blk, g.n); break;
            case 2: class4_kernel<2><<<grid, kJ, 0, s>>>(g.tasks, g.blk, g.n); break;
            case 3: class4_kernel<3><<<grid, kJ, 0, s>>>(g.tasks, g.blk, g.n); break;
            default: class4_kernel<4><<<grid, kJ, 0, s>>>(g.tasks, g.blk, g.n); break;
        }
        return 1;
    }
#define HB_C4DF(WW)                                                                                       \
    switch (ns_tile) {                                                                                    \
        case 4: class4_df_kernel<WW, 4><<<grid, jt, 0, s>>>(g.tasks, g.blk, g.n); break;                 \
        case 8: class4_df_kernel<WW, 8><<<grid, jt, 0, s>>>(g.tasks, g.blk, g.n); break;                 \
        case 12: class4_df_kernel<WW, 12><<<grid, jt, 0, s>>>(g.tasks, g.blk, g.n); break;               \
        case 16: class4_df_kernel<WW, 16><<<grid, jt, 0, s>>>(g.tasks, g.blk, g.n); break;               \
        case 20: class4_df_kernel<WW, 20><<<grid, jt, 0, s>>>(g.tasks, g.blk, g.n); break;               \
        case 24: class4_df_kernel<WW, 24><<<grid, jt, 0, s>>>(g.tasks, g.blk, g.n); break;               \
        case 28: class4_df_kernel<WW, 28><<<grid, jt, 0, s>>>(g.tasks, g.blk, g.n); break;               \
        case 32: class4_df_kernel<WW, 32><<<grid, jt, 0, s>>>(g.tasks, g.blk, g.n); break;               \
        case 40: class4_df_kernel<WW, 40><<<grid, jt, 0, s>>>(g.tasks, g.blk, g.n); break;               \
        case 48: class4_df_kernel<WW, 48><<<grid, jt, 0, s>>>(g.tasks, g.blk, g.n); break;               \
        case 56: class4_df_kernel<WW, 56><<<grid, jt, 0, s>>>(g.tasks, g.blk, g.n); break;               \
        default: class4_df_kernel<WW, 64><<<grid, jt, 0, s>>>(g.tasks, g.blk, g.n); break;               \
    }
    switch (W) {
        case 1: HB_C4DF(1); break;
        case 2: HB_C4DF(2); break;
        case 3: HB_C4DF(3); break;
        default: HB_C4DF(4); break;
    }
#undef HB_C4DF
    return 1;
}

}  // namespace hb
