// K4: class 4, continuum x L2 (Eq. 5), double precision.
//
// For L2 function l and target group g:
//   H~[l][(g n j)] = sum_{m partners of l} c_mn <D_m + j|H|chi_l>
// The classified (m, l) pairs (D_m within a single substitution of chi_l, so
// the (N+1)-electron pair is within a double excitation) are the prototypes;
// each gives, for every continuum orbital j, one or two integrals of the form
// (ab|c j) (plus h_jt for a single excitation), all contiguous in j in the
// (tt|tc) class array, so the 128 threads of a block read them coalesced.
// A block owns one L2 row and 128 continuum orbitals and keeps up to 32
// target states in registers; the CI rows of a batch of partners are staged
// in shared memory.  The prototype values are always evaluated in FP64; the
// rank-1 accumulation over partners is FP64 (plain build) or, in the mixed
// build, double-float FP32 (exact products by FMA, TwoSum accumulation, about
// 44 significant bits), which runs on the FP32 pipes instead of the much
// slower FP64 pipe of this part.
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

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

template <int W, int DF>
__global__ void __launch_bounds__(kJ)
class4_kernel(const C4Task *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    __shared__ double cs[kBatch][kNS];
    __shared__ float ch[kBatch][kNS], cl[kBatch][kNS];
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
        float ahi[kNS], alo[kNS];
#pragma unroll
        for (int n = 0; n < kNS; ++n) { acc[n] = 0.0; ahi[n] = 0.0f; alo[n] = 0.0f; }
        for (int64_t p0 = b; p0 < e; p0 += kBatch) {
            const int cnt = (int)(e - p0 < kBatch ? e - p0 : kBatch);
            __syncthreads();
            if (threadIdx.x < cnt) rs[threadIdx.x] = pairs[p0 + threadIdx.x];
            __syncthreads();
            for (int t = threadIdx.x; t < cnt * kNS; t += kJ) {
                const int i = t / kNS, n = t % kNS;
                const double c = n < nc ? C[(int64_t)rs[i].col * ns + n0 + n] : 0.0;
                if (DF) {
                    const float h = (float)c;
                    ch[i][n] = h;
                    cl[i][n] = (float)(c - (double)h);
                } else {
                    cs[i][n] = c;
                }
            }
            __syncthreads();
            for (int i = 0; i < cnt; ++i) {
                const hb_pair r = rs[i];
                const double y = prototype_value<W>(I, r, dets + (int64_t)r.col * 2 * W, j, cont_spin);
                if (DF) {
                    const float yh = (float)y, yl = (float)(y - (double)yh);
#pragma unroll
                    for (int n = 0; n < kNS; ++n) {
                        const float ph = ch[i][n] * yh;
                        const float pe = fmaf(ch[i][n], yh, -ph);             // exact error of ph
                        const float pl = fmaf(ch[i][n], yl, fmaf(cl[i][n], yh, pe));
                        float sum, err;
                        two_sum(ahi[n], ph, sum, err);
                        ahi[n] = sum;
                        alo[n] = __fadd_rn(alo[n], __fadd_rn(err, pl));
                    }
                } else {
#pragma unroll
                    for (int n = 0; n < kNS; ++n) acc[n] = fma(cs[i][n], y, acc[n]);
                }
            }
        }
        if (jv) {
            double *out = T.Hlc + (int64_t)l * T.ld + T.col_off + jl;
#pragma unroll
            for (int n = 0; n < kNS; ++n)
                if (n < nc) out[(int64_t)(n0 + n) * cn] = DF ? (double)ahi[n] + (double)alo[n] : acc[n];
        }
    }
}

}  // namespace

int class4_ny(int cn) { return (cn + kJ - 1) / kJ; }
int64_t blocks_class4(int n_l2, int cn) { return cn > 0 ? (int64_t)n_l2 * class4_ny(cn) : 0; }

int g_class4(const Grouped<C4Task> &g, int W, int dfloat, cudaStream_t s) {
    if (g.blocks <= 0) return 0;
    const unsigned grid = (unsigned)g.blocks;
#define HB_C4(WW, DD) class4_kernel<WW, DD><<<grid, kJ, 0, s>>>(g.tasks, g.blk, g.n)
    if (dfloat) {
        switch (W) {
            case 1: HB_C4(1, 1); break;
            case 2: HB_C4(2, 1); break;
            case 3: HB_C4(3, 1); break;
            default: HB_C4(4, 1); break;
        }
    } else {
        switch (W) {
            case 1: HB_C4(1, 0); break;
            case 2: HB_C4(2, 0); break;
            case 3: HB_C4(3, 0); break;
            default: HB_C4(4, 0); break;
        }
    }
#undef HB_C4
    return 1;
}

}  // namespace hb
