// Class 4 (Eq. 5) of the mixed build on the 5th-generation tensor cores.
//
// Every classified pair (m, l) of a target determinant and an L2 function
// contributes c_mn y(j) to H~[l][(g n j)], and its prototype value y(j) is a
// signed sum of integral rows that are contiguous in the continuum index j:
//   d = 2 (one substitution): (q h1|h2 j) and/or (q h2|h1 j), one row each,
//   d = 1 (chi_l = D_m + t):  h_jt + sum_{k in D_m} (kk|t j) - sum_{k same spin} (kt|k j).
// Written term by term, an L2 row l is a short GEMM
//   H~[l][n][j] = sum_t  s_t c[m_t][n]  X[x_t][j]
// over its terms t = (integral row x_t, CI row m_t, sign s_t).  Here the two
// operands are gathered rows of tables made once per context:
//   X slices [S][x_rows][jpad]: the (tt|tc) rows, the transposed one-electron
//     rows h[n_to + j][t] and a zero row, split into S bf16 slices with one
//     exponent per continuum orbital j;
//   C slices [S][2 ndet + 1][64] per group: +c, -c and a zero row, one exponent
//     per state n;
// split into balanced base-256 digits, so every slice-pair product of a term
// has the unit 2^(e_j + e_n - 16 - 8 s), at most 2^16 units for s <= 2, and
// the MMAs sum them exactly in FP32 over chunks of at most 256 terms.  The term lists (integral row, signed CI row) per L2 row are
// sized once per plan and written every build from that build's pairs.
//
// Kernel (persistent, one CTA per SM, 13 warps):
//   warp 0     MMA issuer (one thread) and TMEM owner (512 columns: two
//              buffers of 4 accumulators x 64 states, so one work item's
//              epilogue overlaps the next item's MMAs)
//   warps 1-4  producers: cp.async gathers of 32 terms x (128 j + 64 n) per
//              slice into 128-byte-swizzled MN-major tiles, 3 stages
//   warps 5-12 epilogue: TMEM -> double-float (TwoSum for s <= 2) -> FP64
// A work item is (L2 row, tile of 128 continuum orbitals); the tile starts on
// a multiple of 8 orbitals so every 16-byte copy is aligned.  Every wait is
// bounded; on a timeout the kernel records an error and leaves.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "hb_api_internal.cuh"
#include "hb_c4tc.cuh"
#include "hb_df.cuh"
#include "hb_tasks.cuh"
#include "hb_tc.cuh"

namespace hb {

struct C4TC {
    int S = 0;
    int64_t x_rows = 0, x_h0 = 0, x_zero = 0;   // rows: (tt|tc) rows, then h^T rows, then a zero row
    int jpad = 0;
    __nv_bfloat16 *xs = nullptr;
    bool borrowed = false;
    struct Group {
        bool on = false;
        __nv_bfloat16 *cs = nullptr;            // [S][2 ndet + 1][64]
        int64_t c_rows = 0;
        int64_t *term_ptr = nullptr;            // [n_l2 + 1], rows padded to multiples of 32 terms
        std::vector<int64_t> term_ptr_host;
        int2 *terms = nullptr;                  // (x row, C row)
        int64_t n_terms = 0;
    };
    std::vector<Group> g;
};

namespace {

using namespace hb::tc;

constexpr int TKB = 32;          // terms per K block
constexpr int TBM = 128;         // continuum orbitals per tile (TMEM lanes)
constexpr int TNP = 64;          // states per tile (N of the MMA)
constexpr int TSTAGES = 3;
constexpr int TCHUNK_KB = 8;     // K blocks per exact accumulation chunk (256 terms)
constexpr int T_A_SLICE = 2 * (TKB / 8) * 1024;       // 8 KB: two 64-orbital atoms
constexpr int T_B_SLICE = (TKB / 8) * 1024;           // 4 KB: one 64-state atom
constexpr int T_PROD_WARPS = 4, T_EPI_WARPS = 8;
constexpr int T_THREADS = 32 * (1 + T_PROD_WARPS + T_EPI_WARPS);
constexpr int T_PROD_THREADS = 32 * T_PROD_WARPS, T_EPI_THREADS = 32 * T_EPI_WARPS;
constexpr int T_EPI_COLS = TNP / 2;                   // columns per epilogue thread

template <int S>
constexpr int t_stage_bytes() { return S * (T_A_SLICE + T_B_SLICE); }

// double-float accumulation: (hi, lo) += x, exact TwoSum on the high part
__device__ __forceinline__ void df_add(float &hi, float &lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// ------------------------------------------------------------ digit helper
// x = F 2^(e - 8S) with F = round(x 2^(8S - e)) from the FP64 bit pattern
// (|x| < 2^e, so |F| < 2^(8S), at most 2^62 for S <= 6 ... 7); the balanced
// base-256 digits of F are the slices: slice i = d_i 2^(e - 8 - 8i) with
// |d_0| <= 256 and |d_i| <= 128 after it, all exact in bf16 (8 significant
// bits), so six slices carry 48 bits.
__device__ __forceinline__ void slice_value(double x, int e, int S, __nv_bfloat16 *out, int64_t stride) {
    long long F = 0;
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int be = (int)((b >> 52) & 0x7FF);
    if (e > -2000 && be != 0) {
        const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
        const int sh = (be - 1075) + 8 * S - e;
        long long f;
        if (sh >= 0) f = m << sh;           // sh <= 8S - 53 + 1 <= 0 for S <= 6
        else if (sh > -63) f = (m + (1ll << (-sh - 1))) >> (-sh);
        else f = 0;
        F = (b >> 63) ? -f : f;
    }
    for (int i = 0; i < S; ++i) {
        const int sh = 8 * (S - 1 - i);
        const long long d = sh > 0 ? ((F + (1ll << (sh - 1))) >> sh) : F;
        F -= d << sh;
        out[(int64_t)i * stride] = __float2bfloat16_rn(e > -2000 ? ldexpf((float)d, e - 8 - 8 * i) : 0.0f);
    }
}

__device__ __forceinline__ int exp_of(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int be = (int)((b >> 52) & 0x7FF);
    return be == 0 ? -2000 : be - 1022;         // |x| < 2^e
}

__global__ void fill_int_kernel(int *x, int n, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// value of table row r at column j: (tt|tc) rows, then h^T rows, then zero
__device__ __forceinline__ double x_value(const double *tttc, const double *h, int64_t n_tc_rows, int n_to, int n_co,
                                          int n_orb, int64_t r, int j) {
    if (j >= n_co) return 0.0;
    if (r < n_tc_rows) return tttc[r * n_co + j];
    const int64_t t = r - n_tc_rows;
    if (t < n_to) return h[(int64_t)(n_to + j) * n_orb + t];
    return 0.0;
}

// column exponents of the integral table: blocks of 64 rows, threads over j
__global__ void x_colexp_kernel(const double *tttc, const double *h, int64_t n_tc_rows, int n_to, int n_co, int n_orb,
                                int64_t x_rows, int *e) {
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    for (int j = threadIdx.x; j < n_co; j += blockDim.x) {
        int m = -2000;
        for (int64_t r = r0; r < r0 + 64 && r < x_rows; ++r) m = max(m, exp_of(x_value(tttc, h, n_tc_rows, n_to, n_co, n_orb, r, j)));
        if (m > -2000) atomicMax(e + j, m);
    }
}

__global__ void x_slice_kernel(const double *tttc, const double *h, int64_t n_tc_rows, int n_to, int n_co, int n_orb,
                               int64_t x_rows, int jpad, int S, const int *e, __nv_bfloat16 *xs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= x_rows * jpad) return;
    const int64_t r = i / jpad;
    const int j = (int)(i % jpad);
    const double v = x_value(tttc, h, n_tc_rows, n_to, n_co, n_orb, r, j);
    slice_value(v, j < n_co ? e[j] : -2000, S, xs + r * jpad + j, x_rows * jpad);
}

// CI slices of one group: rows m (+c), ndet + m (-c), 2 ndet (zero); 64 columns
__global__ void c_colexp_kernel(const double *C, int ndet, int ns, int *e) {
    const int n = threadIdx.x;
    if (n >= ns) return;
    int m = -2000;
    for (int64_t r = (int64_t)blockIdx.x * 256; r < (int64_t)(blockIdx.x + 1) * 256 && r < ndet; ++r)
        m = max(m, exp_of(C[r * ns + n]));
    if (m > -2000) atomicMax(e + n, m);
}

__global__ void c_slice_kernel(const double *C, int ndet, int ns, int S, const int *e, __nv_bfloat16 *cs) {
    const int64_t r = blockIdx.x;                 // 0 .. 2 ndet
    const int n = threadIdx.x;                    // 0 .. 63
    const int64_t rows = 2 * (int64_t)ndet + 1;
    double v = 0.0;
    if (n < ns && r < 2 * (int64_t)ndet) {
        const double c = C[(r % ndet) * ns + n];
        v = r < ndet ? c : -c;
    }
    slice_value(v, n < ns ? e[n] : -2000, S, cs + r * TNP + n, rows * TNP);
}

// ------------------------------------------------------------- term lists
// The terms of one pair (the prototype's integral rows and signs), written to
// out[0..) when WRITE; returns their number.
template <bool WRITE>
__device__ __forceinline__ int pair_terms(const hb_pair &r, const uint64_t *__restrict__ D, int W, int n_to,
                                          int cont_spin, int ndet, int64_t x_h0, int2 *out) {
    const int sb = 64 * W;
    const int m = r.col;
    auto crow = [&](int sign) { return sign * r.phase > 0 ? m : ndet + m; };
    int n = 0;
    if (r.degree == 1) {
        // chi = D + t (spin cont_spin): h_jt + sum_k (jt|kk) - sum_{k same spin} (jk|kt)
        const int t = r.hole[0] % sb;
        if (WRITE) out[n] = make_int2((int)(x_h0 + t), crow(1));
        ++n;
        for (int w = 0; w < 2 * W; ++w) {
            uint64_t x = D[w];
            const int s = w / W;
            while (x) {
                const int k = 64 * (w % W) + __ffsll((long long)x) - 1;
                x &= x - 1;
                if (WRITE) out[n] = make_int2((int)(pair_idx(k, k) * n_to + t), crow(1));
                ++n;
                if (s == cont_spin) {
                    if (WRITE) out[n] = make_int2((int)(pair_idx(k, t) * n_to + k), crow(-1));
                    ++n;
                }
            }
        }
        return n;
    }
    // degree 2: holes h1 < h2 in chi, particles {q, continuum} in D + j
    const int h1 = r.hole[0], h2 = r.hole[1], q = r.part[0];
    const int kq = 2 * q, kv = cont_spin == 0 ? 2 * 64 * W - 1 : 2 * 128 * W - 1;
    const int s1 = h1 / sb, s2 = h2 / sb, sq = q / sb;
    const int o1 = h1 % sb, o2 = h2 % sb, oq = q % sb;
    bool dir, exc;
    int64_t xd, xe;
    if (kq < kv) {
        dir = sq == s1 && cont_spin == s2;   // (q h1|j h2)
        exc = sq == s2 && cont_spin == s1;   // (q h2|j h1)
        xd = pair_idx(oq, o1) * n_to + o2;
        xe = pair_idx(oq, o2) * n_to + o1;
    } else {
        dir = cont_spin == s1 && sq == s2;   // (j h1|q h2)
        exc = cont_spin == s2 && sq == s1;   // (j h2|q h1)
        xd = pair_idx(oq, o2) * n_to + o1;
        xe = pair_idx(oq, o1) * n_to + o2;
    }
    if (dir) {
        if (WRITE) out[n] = make_int2((int)xd, crow(1));
        ++n;
    }
    if (exc) {
        if (WRITE) out[n] = make_int2((int)xe, crow(-1));
        ++n;
    }
    return n;
}

// terms of each L2 row (a warp per row), padded to a multiple of TKB, into cnt[l + 1]
__global__ void term_count_kernel(const hb_pair *__restrict__ pairs, const int64_t *__restrict__ row_ptr, int n_l2,
                                  const uint64_t *__restrict__ dets, int W, int n_to, int cont_spin, int ndet,
                                  int64_t *cnt) {
    const int lane = threadIdx.x & 31;
    const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (l >= n_l2) return;
    int64_t c = 0;
    for (int64_t k = row_ptr[l] + lane; k < row_ptr[l + 1]; k += 32) {
        const hb_pair r = pairs[k];
        c += pair_terms<false>(r, dets + (int64_t)r.col * 2 * W, W, n_to, cont_spin, ndet, 0, nullptr);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if (lane == 0) cnt[l + 1] = (c + TKB - 1) / TKB * TKB;
}

// the terms of each L2 row in pair order, then zero terms up to the padded count
__global__ void term_fill_kernel(const C4FTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const C4FTask T = tasks[ti];
    const int lane = threadIdx.x & 31;
    const int l = (int)(blockIdx.x - blk[ti]) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (l >= T.n_l2) return;
    int64_t pos = T.term_ptr[l];
    const int64_t end = T.term_ptr[l + 1];
    const int64_t b = T.row_ptr[l], e = T.row_ptr[l + 1];
    for (int64_t k0 = b; k0 < e; k0 += 32) {
        const int64_t k = k0 + lane;
        hb_pair r;
        int c = 0;
        if (k < e) {
            r = T.pairs[k];
            c = pair_terms<false>(r, T.dets + (int64_t)r.col * 2 * T.W, T.W, T.n_to, T.cont_spin, T.ndet, T.x_h0, nullptr);
        }
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        const int excl = incl - c;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (k < e && pos + excl + c <= end)
            pair_terms<true>(r, T.dets + (int64_t)r.col * 2 * T.W, T.W, T.n_to, T.cont_spin, T.ndet, T.x_h0,
                             T.terms + pos + excl);
        pos += total;
    }
    for (int64_t p = pos + lane; p < end; p += 32) T.terms[p] = make_int2((int)T.x_zero, 2 * T.ndet);
}

// ------------------------------------------------------------- the kernel
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 128-byte-swizzled MN-major descriptor: atoms of 64 MN elements x 8 K rows
// (1 KB); LBO = distance between atoms along MN, SBO = between 8-row K groups.
__device__ __forceinline__ uint64_t desc_mn(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ C4Item load_item(const C4Item *__restrict__ items, int n_items, int item) {
    C4Item r;
    if (item < n_items) r = items[item];
    else r = C4Item{0, 0, 0, 0, 0};
    return r;
}

// Fold one chunk of the four accumulators (T_EPI_COLS columns at this thread's
// lane; accumulator s at column offset s * TNP) into the double-float sums.
template <int S>
__device__ __forceinline__ void drain_c4(uint32_t tbase, float (&hi)[T_EPI_COLS], float (&lo)[T_EPI_COLS]) {
    constexpr int n_acc = S < 4 ? S : 4;
#pragma unroll
    for (int c0 = 0; c0 < T_EPI_COLS; c0 += 16) {
        uint32_t v[16], w[16];
        tmem_ld16_async(tbase + c0, v);
        if (n_acc > 1) tmem_ld16_async(tbase + TNP + c0, w);
        tmem_wait_ld();
        tmem_regs_ready(v);
        if (n_acc > 1) tmem_regs_ready(w);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            df_add(hi[c0 + i], lo[c0 + i], __uint_as_float(v[i]));
            if (n_acc > 1) df_add(hi[c0 + i], lo[c0 + i], __uint_as_float(w[i]));
        }
        if (n_acc > 2) {
            tmem_ld16_async(tbase + 2 * TNP + c0, v);
            if (n_acc > 3) tmem_ld16_async(tbase + 3 * TNP + c0, w);
            tmem_wait_ld();
            tmem_regs_ready(v);
            if (n_acc > 3) tmem_regs_ready(w);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                df_add(hi[c0 + i], lo[c0 + i], __uint_as_float(v[i]));
                if (n_acc > 3) lo[c0 + i] = __fadd_rn(lo[c0 + i], __uint_as_float(w[i]));
            }
        }
    }
}

template <int S>
__global__ void __launch_bounds__(T_THREADS, 1)
class4_tc_kernel(const C4TTask *__restrict__ tasks, const C4Item *__restrict__ items, int n_items, int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int STAGE = t_stage_bytes<S>();
    uint64_t *full_bar = (uint64_t *)(base + TSTAGES * STAGE);
    uint64_t *empty_bar = full_bar + TSTAGES;
    uint64_t *acc_full = empty_bar + TSTAGES;   // [2]
    uint64_t *acc_empty = acc_full + 2;         // [2]
    uint64_t *final_bar = acc_empty + 2;
    uint32_t *tmem_slot = (uint32_t *)(final_bar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < TSTAGES; ++i) { mbar_init(&full_bar[i], T_PROD_THREADS); mbar_init(&empty_bar[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&acc_full[i], 1); mbar_init(&acc_empty[i], T_EPI_THREADS); }
        mbar_init(final_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = instr_desc_bf16(TBM, TNP) | (1u << 15) | (1u << 16);   // both operands MN-major
            const uint32_t sbase = smem_u32(base);
            bool ok = true;
            int G = 0, it = 0;
            int cnt[2] = {0, 0};                // accumulator hand-overs per buffer
            C4Item nx = load_item(items, n_items, blockIdx.x);
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x, ++it) {
                const C4Item cur = nx;
                nx = load_item(items, n_items, item + gridDim.x);   // next record in flight
                const int nkb = cur.nkb;
                const int buf = it & 1;
                for (int kb0 = 0; kb0 < nkb && ok; kb0 += TCHUNK_KB) {
                    if (cnt[buf] > 0) ok = mbar_wait(&acc_empty[buf], (cnt[buf] - 1) & 1, err, 21);
                    if (!ok) break;
                    tc_fence_after();
                    uint32_t fresh = 0xFu;
                    const int kb1 = min(nkb, kb0 + TCHUNK_KB);
                    for (int kb = kb0; kb < kb1 && ok; ++kb, ++G) {
                        const int q = G % TSTAGES;
                        ok = mbar_wait(&full_bar[q], (G / TSTAGES) & 1, err, 22);
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t sa = sbase + q * STAGE, sbb = sa + S * T_A_SLICE;
#pragma unroll
                        for (int ks = 0; ks < TKB / 16; ++ks) {
#pragma unroll
                            for (int i = 0; i < S; ++i) {
#pragma unroll
                                for (int l2 = 0; l2 < S; ++l2) {
                                    if (i + l2 >= S) continue;
                                    const int s = i + l2 < 3 ? i + l2 : 3;
                                    const uint64_t ad = desc_mn(sa + i * T_A_SLICE + ks * 2048, T_A_SLICE / 2, 1024);
                                    const uint64_t bd = desc_mn(sbb + l2 * T_B_SLICE + ks * 2048, T_A_SLICE / 2, 1024);
                                    const uint32_t acc = (fresh >> s) & 1u ? 0u : 1u;
                                    mma_bf16(tmem + buf * 256 + s * TNP, ad, bd, idesc, acc);
                                    fresh &= ~(1u << s);
                                }
                            }
                        }
                        mma_commit(&empty_bar[q]);          // the stage is free once these MMAs complete
                    }
                    if (ok) mma_commit(&acc_full[buf]);
                    ++cnt[buf];
                }
            }
            mma_commit(final_bar);
            mbar_wait(final_bar, 0, err, 23);
        }
    } else if (warp <= T_PROD_WARPS) {
        // ----------------------------------------------------------- producers
        // Thread pt copies, in every slice, the 16-byte chunks (tt, ch) with
        // tt * 16 + ch = pt + 128 u (A, u < 4) and tt * 8 + ch = pt + 128 u
        // (B, u < 2): six terms per stage, read one stage ahead.
        const int pt = threadIdx.x - 32;          // 0 .. T_PROD_THREADS-1
        constexpr int NA = TKB * 16 / T_PROD_THREADS, NB = TKB * 8 / T_PROD_THREADS;
        const uint32_t sbase = smem_u32(base);
        bool ok = true;
        int G = 0;
        // the K blocks of this CTA in order: (item record, block) with the next one's terms in flight
        int item = blockIdx.x, kb = 0;
        C4Item cur = load_item(items, n_items, item);
        while (item < n_items && cur.nkb == 0) { item += gridDim.x; cur = load_item(items, n_items, item); }
        int2 ta[NA], tb[NB];
        auto load_terms = [&](const C4Item &it, int k, int2 (&xa)[NA], int2 (&xb)[NB]) {
            const int2 *terms = tasks[it.ti].terms + it.t0 + (int64_t)k * TKB;
#pragma unroll
            for (int u = 0; u < NA; ++u) xa[u] = __ldg(terms + (pt + T_PROD_THREADS * u) / 16);
#pragma unroll
            for (int u = 0; u < NB; ++u) xb[u] = __ldg(terms + (pt + T_PROD_THREADS * u) / 8);
        };
        if (item < n_items) load_terms(cur, 0, ta, tb);
        while (item < n_items && ok) {
            // the next K block of this CTA (possibly of a later item) and its terms
            int nitem = item, nkb = kb + 1;
            C4Item nxt = cur;
            if (nkb >= cur.nkb) {
                nkb = 0;
                do {
                    nitem += gridDim.x;
                    nxt = load_item(items, n_items, nitem);
                } while (nitem < n_items && nxt.nkb == 0);
            }
            int2 na[NA], nb[NB];
            if (nitem < n_items) load_terms(nxt, nkb, na, nb);
            const C4TTask &T = tasks[cur.ti];
            const int j0 = T.j0 + cur.jt * TBM;
            const __nv_bfloat16 *cs = (const __nv_bfloat16 *)T.cs;
            const __nv_bfloat16 *xs = (const __nv_bfloat16 *)T.xs;
            const int64_t c_rows = T.c_rows, x_rows = T.x_rows;
            const int jpad = T.jpad;
            const int q = G % TSTAGES;
            if (G >= TSTAGES) ok = mbar_wait(&empty_bar[q], ((G / TSTAGES) - 1) & 1, err, 24);
            if (!ok) break;
            const uint32_t sa = sbase + q * STAGE, sbb = sa + S * T_A_SLICE;
#pragma unroll
            for (int i = 0; i < S; ++i) {
#pragma unroll
                for (int u = 0; u < NA; ++u) {
                    const int pidx = pt + T_PROD_THREADS * u;
                    const int tt = pidx / 16, ch = pidx % 16;
                    const int j = j0 + ch * 8;
                    const uint32_t off = (uint32_t)(i * T_A_SLICE + (ch >> 3) * (T_A_SLICE / 2) + (tt >> 3) * 1024 +
                                                    (tt & 7) * 128 + (((ch & 7) ^ (tt & 7)) << 4));
                    const bool in = j + 8 <= jpad;
                    const __nv_bfloat16 *src = xs + ((int64_t)i * x_rows + ta[u].x) * jpad + (in ? j : 0);
                    cp_async16(sa + off, src, in ? 16u : 0u);
                }
#pragma unroll
                for (int u = 0; u < NB; ++u) {
                    const int pidx = pt + T_PROD_THREADS * u;
                    const int tt = pidx / 8, ch = pidx % 8;
                    const uint32_t off = (uint32_t)(i * T_B_SLICE + (tt >> 3) * 1024 + (tt & 7) * 128 + ((ch ^ (tt & 7)) << 4));
                    cp_async16(sbb + off, cs + ((int64_t)i * c_rows + tb[u].y) * TNP + ch * 8, 16u);
                }
            }
            cp_async_commit();
            if (G > 1) {
                // the copies of two stages back have landed: publish them to the
                // tensor cores (three stages of copies in flight per thread)
                cp_async_wait2();
                fence_async_smem();
                mbar_arrive(&full_bar[(G - 2) % TSTAGES]);
            }
            ++G;
            item = nitem;
            kb = nkb;
            cur = nxt;
#pragma unroll
            for (int u = 0; u < NA; ++u) ta[u] = na[u];
#pragma unroll
            for (int u = 0; u < NB; ++u) tb[u] = nb[u];
        }
        // the last two stages
        if (ok && G > 1) {
            cp_async_wait1();
            fence_async_smem();
            mbar_arrive(&full_bar[(G - 2) % TSTAGES]);
        }
        cp_async_wait0();
        if (ok && G > 0) {
            fence_async_smem();
            mbar_arrive(&full_bar[(G - 1) % TSTAGES]);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - 1 - T_PROD_WARPS;   // 0 .. 7
        const int qd = warp & 3;                  // TMEM lane quadrant of this warp
        const int col0 = (ew >> 2) * T_EPI_COLS;
        const int row = qd * 32 + lane;
        bool ok = true;
        int it = 0;
        int cnt[2] = {0, 0};
        C4Item nx = load_item(items, n_items, blockIdx.x);
        for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x, ++it) {
            const C4Item cur = nx;
            nx = load_item(items, n_items, item + gridDim.x);
            const C4TTask &T = tasks[cur.ti];
            const int nkb = cur.nkb;
            const int buf = it & 1;
            float hi[T_EPI_COLS], lo[T_EPI_COLS];
#pragma unroll
            for (int c = 0; c < T_EPI_COLS; ++c) { hi[c] = 0.0f; lo[c] = 0.0f; }
            for (int kb0 = 0; kb0 < nkb && ok; kb0 += TCHUNK_KB) {
                ok = mbar_wait(&acc_full[buf], cnt[buf] & 1, err, 25);
                if (!ok) break;
                tc_fence_after();
                drain_c4<S>(tmem + ((uint32_t)(qd * 32) << 16) + buf * 256 + col0, hi, lo);
                tc_fence_before();
                mbar_arrive(&acc_empty[buf]);
                ++cnt[buf];
            }
            if (!ok) break;
            const int j = T.j0 + cur.jt * TBM + row;
            if (j >= T.cf && j < T.cf + T.cn) {
                double *out = T.Hlc + (int64_t)cur.l * T.ld + T.col_off + (j - T.cf);
#pragma unroll
                for (int c = 0; c < T_EPI_COLS; ++c) {
                    const int n = col0 + c;
                    if (n < T.ns) out[(int64_t)n * T.cn] = df_to_double(hi[c], lo[c]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

template <int S>
cudaError_t set_attr() {
    return cudaFuncSetAttribute(class4_tc_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TSTAGES * t_stage_bytes<S>() + 2048);
}

int sm_count_c4() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 1;
    }
    return n;
}

int c4_fail(hb_ctx *ctx, int rc, const std::string &msg) {
    ctx->err = "class-4 tensor operands: " + msg;
    return rc;
}

template <class T>
cudaError_t c4_alloc(hb_ctx *ctx, T **p, size_t n) {
    cudaError_t e = dmalloc_n(ctx, p, n);
    if (e == cudaSuccess) ctx->dev_bytes += sizeof(T) * (n ? n : 1);
    return e;
}

}  // namespace

// ------------------------------------------------------------------ host
bool c4tc_group_on(const hb_ctx *ctx, int g) {
    const C4TC *c = (const C4TC *)ctx->c4tc;
    return c && g < (int)c->g.size() && c->g[g].on;
}

int c4tc_min_states(const hb_ctx *ctx) { return ctx->c4_path == 2 ? 1 : 32; }

int c4tc_prepare(hb_ctx *ctx, int S, cudaStream_t s) {
    if (ctx->c4tc) return HB_OK;
    if (S < 2 || S > 6) return c4_fail(ctx, HB_ERR_INVALID_ARG, "slices must be 2..6");
    bool any = false;      // nothing to make unless some group takes the tensor-core path
    for (int g = 0; g < ctx->n_groups; ++g) {
        const GroupInfo &Gi = ctx->groups[g];
        any = any || (Gi.ns >= c4tc_min_states(ctx) && Gi.ns <= TNP && Gi.cn > 0 && Gi.ndet > 0 && ctx->n_l2 > 0);
    }
    if (!any) return HB_OK;
    C4TC *c = new C4TC();
    ctx->c4tc = c;
    c->S = S;
    const int64_t n_tc_rows = ctx->Pt * ctx->n_to;
    c->x_h0 = n_tc_rows;
    c->x_zero = n_tc_rows + ctx->n_to;
    c->x_rows = c->x_zero + 1;
    c->jpad = (ctx->n_co + 7) / 8 * 8;
    if (c->x_rows >= (1ll << 31)) return c4_fail(ctx, HB_ERR_INVALID_ARG, "integral table too large");
    cudaError_t e = cudaSuccess;
    if (ctx->base) {
        int rc = c4tc_prepare(ctx->base, S, s);
        if (rc != HB_OK) return c4_fail(ctx, rc, ctx->base->err);
        const C4TC *b = (const C4TC *)ctx->base->c4tc;
        c->xs = b->xs;
        c->borrowed = true;
    } else {
        int *ex = nullptr;
        e = dmalloc_n(ctx, &ex, (size_t)(ctx->n_co > 0 ? ctx->n_co : 1));
        if (e == cudaSuccess) e = c4_alloc(ctx, &c->xs, (size_t)S * c->x_rows * c->jpad);
        if (e != cudaSuccess) {
            dfree(ctx, ex);
            return c4_fail(ctx, HB_ERR_OOM, cudaGetErrorString(e));
        }
        if (ctx->n_co > 0) {
            fill_int_kernel<<<(ctx->n_co + 255) / 256, 256, 0, s>>>(ex, ctx->n_co, -2000);
            x_colexp_kernel<<<(unsigned)((c->x_rows + 63) / 64), 128, 0, s>>>(ctx->tttc, ctx->h, n_tc_rows, ctx->n_to,
                                                                           ctx->n_co, ctx->n_orb, c->x_rows, ex);
        }
        x_slice_kernel<<<(unsigned)((c->x_rows * c->jpad + 255) / 256), 256, 0, s>>>(ctx->tttc, ctx->h, n_tc_rows, ctx->n_to, ctx->n_co, ctx->n_orb, c->x_rows,
                                            c->jpad, S, ex, c->xs);
        e = cudaStreamSynchronize(s);
        dfree(ctx, ex);
        if (e != cudaSuccess) return c4_fail(ctx, HB_ERR_CUDA, cudaGetErrorString(e));
    }
    e = set_attr<2>();
    if (e == cudaSuccess) e = set_attr<3>();
    if (e == cudaSuccess) e = set_attr<4>();
    if (e == cudaSuccess) e = set_attr<5>();
    if (e == cudaSuccess) e = set_attr<6>();
    if (e != cudaSuccess) return c4_fail(ctx, HB_ERR_CUDA, cudaGetErrorString(e));
    c->g.resize(ctx->n_groups);
    for (int g = 0; g < ctx->n_groups; ++g) {
        const GroupInfo &Gi = ctx->groups[g];
        C4TC::Group &cg = c->g[g];
        if (Gi.ns < c4tc_min_states(ctx) || Gi.ns > TNP || Gi.cn < 1 || ctx->n_l2 < 1 || Gi.ndet < 1) continue;
        const GroupL2 &L = ctx->gl2[g];
        const uint64_t *dg = ctx->dets + Gi.det_off;
        // CI slices
        cg.c_rows = 2 * (int64_t)Gi.ndet + 1;
        int *en = nullptr;
        e = dmalloc_n(ctx, &en, (size_t)TNP);
        if (e == cudaSuccess) e = c4_alloc(ctx, &cg.cs, (size_t)S * cg.c_rows * TNP);
        if (e == cudaSuccess) e = c4_alloc(ctx, &cg.term_ptr, (size_t)ctx->n_l2 + 1);
        if (e != cudaSuccess) {
            dfree(ctx, en);
            return c4_fail(ctx, HB_ERR_OOM, cudaGetErrorString(e));
        }
        fill_int_kernel<<<1, TNP, 0, s>>>(en, TNP, -2000);
        c_colexp_kernel<<<(Gi.ndet + 255) / 256, TNP, 0, s>>>(ctx->ci + Gi.ci_off, Gi.ndet, Gi.ns, en);
        c_slice_kernel<<<(unsigned)cg.c_rows, TNP, 0, s>>>(ctx->ci + Gi.ci_off, Gi.ndet, Gi.ns, S, en, cg.cs);
        // the pairs of this build order, then the padded term counts per L2 row
        k1_fill_pairs(ctx->l2, ctx->n_l2, dg, Gi.ndet, ctx->W, 1, ctx->cont_spin, 2, 0, L.rowptr, L.pairs, s);
        cudaMemsetAsync(cg.term_ptr, 0, sizeof(int64_t), s);
        term_count_kernel<<<(ctx->n_l2 + 7) / 8, 256, 0, s>>>(L.pairs, L.rowptr, ctx->n_l2, dg, ctx->W, ctx->n_to,
                                                               ctx->cont_spin, Gi.ndet, cg.term_ptr);
        std::vector<int64_t> h(ctx->n_l2 + 1);
        e = cudaMemcpyAsync(h.data(), cg.term_ptr, sizeof(int64_t) * h.size(), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        dfree(ctx, en);
        if (e != cudaSuccess) return c4_fail(ctx, HB_ERR_CUDA, cudaGetErrorString(e));
        for (size_t i = 1; i < h.size(); ++i) h[i] += h[i - 1];
        cg.n_terms = h.back();
        cg.term_ptr_host = h;
        e = cudaMemcpyAsync(cg.term_ptr, h.data(), sizeof(int64_t) * h.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = c4_alloc(ctx, &cg.terms, (size_t)cg.n_terms);
        // valid rows (0, 0) until the first build writes the lists
        if (e == cudaSuccess) e = cudaMemsetAsync(cg.terms, 0, sizeof(int2) * (cg.n_terms ? cg.n_terms : 1), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return c4_fail(ctx, HB_ERR_OOM, cudaGetErrorString(e));
        cg.on = true;
    }
    return HB_OK;
}

void c4tc_items(const hb_ctx *ctx, int g, int ti, std::vector<C4Item> *items) {
    const C4TC &c = *(const C4TC *)ctx->c4tc;
    const C4TC::Group &cg = c.g[g];
    const GroupInfo &Gi = ctx->groups[g];
    const int j0 = Gi.cf & ~7;
    const int n_jt = (Gi.cf + Gi.cn - j0 + TBM - 1) / TBM;
    for (int l = 0; l < ctx->n_l2; ++l) {
        const int64_t t0 = cg.term_ptr_host[l];
        const int nkb = (int)((cg.term_ptr_host[l + 1] - t0) / TKB);
        for (int jt = 0; jt < n_jt; ++jt) items->push_back(C4Item{t0, ti, l, jt, nkb});
    }
}

void c4tc_tasks(const hb_ctx *ctx, int g, double *Hlc, C4FTask *fill, int64_t *fill_blocks, C4TTask *tc,
                int64_t *tc_items) {
    const C4TC &c = *(const C4TC *)ctx->c4tc;
    const C4TC::Group &cg = c.g[g];
    const GroupInfo &Gi = ctx->groups[g];
    const GroupL2 &L = ctx->gl2[g];
    *fill = C4FTask{L.pairs, L.rowptr, ctx->n_l2, ctx->dets + Gi.det_off, ctx->W, ctx->n_to, ctx->cont_spin,
                    Gi.ndet, c.x_h0, c.x_zero, cg.term_ptr, cg.terms};
    *fill_blocks = (ctx->n_l2 + 7) / 8;
    const int j0 = Gi.cf & ~7;
    const int n_jt = (Gi.cf + Gi.cn - j0 + TBM - 1) / TBM;
    *tc = C4TTask{c.xs, c.x_rows, c.jpad, cg.term_ptr, cg.terms, ctx->n_l2, n_jt, j0, Gi.cf, Gi.cn, Gi.ns, cg.cs,
                  cg.c_rows, Gi.row_off, ctx->Dc, Hlc};
    *tc_items = (int64_t)ctx->n_l2 * n_jt;
}

int g_c4fill(const Grouped<C4FTask> &g, cudaStream_t s) {
    if (g.blocks <= 0) return 0;
    term_fill_kernel<<<(unsigned)g.blocks, 256, 0, s>>>(g.tasks, g.blk, g.n);
    return 1;
}

int g_c4tc(const Grouped<C4TTask> &g, const C4Item *items, int n_items, int S, int *err, cudaStream_t s) {
    if (n_items <= 0 || g.n <= 0) return 0;
    const unsigned grid = (unsigned)std::min(n_items, sm_count_c4());
#define HB_C4TC(SS)                                                                                                   \
    class4_tc_kernel<SS><<<grid, T_THREADS, TSTAGES * t_stage_bytes<SS>() + 2048, s>>>(g.tasks, items, n_items, err)
    switch (S) {
        case 2: HB_C4TC(2); break;
        case 3: HB_C4TC(3); break;
        case 4: HB_C4TC(4); break;
        case 5: HB_C4TC(5); break;
        default: HB_C4TC(6); break;
    }
#undef HB_C4TC
    return 1;
}

void release_c4tc(hb_ctx *ctx) {
    C4TC *c = (C4TC *)ctx->c4tc;
    if (!c) return;
    if (!c->borrowed) dfree(ctx, c->xs);
    for (auto &g : c->g) {
        dfree(ctx, g.cs);
        dfree(ctx, g.term_ptr);
        dfree(ctx, g.terms);
    }
    delete c;
    ctx->c4tc = nullptr;
}

}  // namespace hb
