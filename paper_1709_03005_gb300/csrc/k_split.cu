// Split-precision expansion (Eq. 7) on the 5th-generation tensor cores.
//
//   out[(j,j'), (n,n')] = sum_k P[(j,j')][k] * A[(n,n')][k]
//
// Both FP64 operands are split row by row into S bf16 slices (an error-free
// splitting in the manner of Ozaki, Ogita, Oishi & Rump 2012): with 2^e the
// smallest power of two above the row's largest magnitude,
//   slice 0 = rint(x 2^{7-e}) 2^{e-7},  |integer| <= 128,
//   slice i = rint(r_i 2^{7+7i-e}) 2^{e-7-7i}, |integer| <= 64  (i >= 1),
// with r_i the remainder after slices 0..i-1, so S slices carry 7S bits.  The
// row exponent is folded into the slice values, so every product of slice i of
// a panel row with slice l of a coefficient row is an integer multiple of the
// same unit 2^{e_row + e_col - 14 - 7(i+l)}.  The products with the same
// s = i + l are summed by tcgen05.mma (kind::f16, bf16 inputs, FP32
// accumulation in tensor memory) in K-chunks of 512: there every partial sum
// stays below 2^24 units, so the FP32 accumulation is exact.  Separate TMEM
// accumulators hold s = 0, 1, 2 and one holds s >= 3 (its rounding is below
// 2^-45 of the result).  The epilogue drains the accumulators after each
// chunk; the MMAs of the next chunk wait for that drain.  After each chunk the
// epilogue warps fold the four accumulators into a double-float running sum
// (TwoSum for s <= 2), and at the end write it as FP64.  Pairs with i + l >= S are dropped (below 2^-7S relative).
//
// Kernel structure (one CTA per 128 x 128 output tile, 10 warps):
//   warp 0  TMA producer: per 32-wide K stage and slice, one panel tile
//           (128 x 32) and one coefficient tile (128 x 32), 64-byte swizzle,
//           each slice in its own shared-memory slot with full/empty mbarriers
//           so the MMAs start as slices land and slots refill as they free;
//           two full sets of slots (six slices), so a stage loads while the
//           one before it is multiplied
//   warp 1  MMA issuer (one elected thread), TMEM allocation owner
//   warps 2-9 epilogue: TMEM -> registers, double-float accumulation, FP64 out
//           (two warps per TMEM lane quadrant, 64 columns each)
// Every mbarrier wait is bounded; on a timeout the kernel records an error,
// drains its own copies and MMAs, frees TMEM and returns.
//
// Rows with j == j' carry h_jj and the delta_jj' E term and so have a wide
// dynamic range; the mixed kernel skips them and an FP64 kernel computes them.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "hb_api_internal.cuh"
#include "hb_split.cuh"
#include "hb_df.cuh"
#include "hb_tc.cuh"

namespace hb {

struct MixedState {
    int slices = 6;
    int64_t panel_rows = 0;
    __nv_bfloat16 *panel_slices = nullptr;   // [S][Kpad/64][n_co*n_co][64]
    bool panel_ready = false;
    bool borrowed_panel = false;
    // [stage width 32, 64][box of 8 x 16, 16 x 8, 32 x 4 continuum pairs (j' x j)]
    CUtensorMap tm_panel[2][3];
    float2 *pdiag = nullptr;                  // diagonal panel rows (j, j) as float pairs [n_co][Kpad]
};

}  // namespace hb

using namespace hb;

namespace {

using namespace hb::tc;

constexpr int BM = 128, BN = 128, BKB = 64;  // tile rows, tile cols, K per block (one 128-B swizzle row)
constexpr int KCHUNK = 512;                  // exact FP32 accumulation span
constexpr int MAXS = 6;
constexpr int A_TILE = BM * BKB * 2;         // 16 KB
constexpr int B_TILE = BN * BKB * 2;         // 16 KB
constexpr int SLOT = A_TILE + B_TILE;        // one slice of one K block (S slots in shared memory)
constexpr int TMEM_COLS = 512;               // 4 accumulators x 128 columns
constexpr int EPI_WARPS = 8;                 // 2 per TMEM lane quadrant
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int EPI_COLS = BN / 2;             // columns per epilogue thread
constexpr int NTHREADS = 64 + EPI_THREADS;

// The expansion kernel's K pipeline: stages of KS = 32 K (64-byte operand
// rows, 64-byte swizzle) or 64 K (128-byte rows and swizzle), and as many full
// sets of S slots as fit 192 KB, so the copies of the next stages are in
// flight while the stages before them are multiplied.  With one set (64-K
// stages and 128 columns) odd stages use the slots in the order in which the
// even ones free them (slot_of).  Its tile is 128 continuum pairs x TBN
// columns (state pairs), TBN = 32, 64 or 128 chosen per merged block from its
// column count; with TBN <= 64 the four accumulators are double-buffered in
// tensor memory, so the MMAs of the next chunk run while the epilogue drains
// the last one.  64-K stages serve 128-column tiles over long K (fewer waits
// and copies per K), 32-K stages the rest (deeper prefetch).
constexpr int XBUDGET = 192 * 1024;          // shared memory of the slots
constexpr int XBARS = 24;                    // full and empty barriers: slots at most
constexpr int kK64Blocks = 32;               // 64-K stages from this many 64-wide K blocks up
__host__ __device__ constexpr int xa_tile(int ks) { return BM * ks * 2; }
// one slice of one stage: panel tile, then coefficient tile (multiples of 1 KB)
__host__ __device__ constexpr int xslot(int tbn, int ks) { return (BM + tbn) * ks * 2; }
__host__ __device__ constexpr int xsets(int S, int tbn, int ks) {
    return XBUDGET / (S * xslot(tbn, ks)) < 4 ? XBUDGET / (S * xslot(tbn, ks)) : 4;
}
__host__ __device__ constexpr int xacc_bufs(int tbn) { return 8 * tbn <= 512 ? 2 : 1; }
__host__ __device__ constexpr int xtmem_cols(int tbn) { return xacc_bufs(tbn) * 4 * tbn; }

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *tm, uint64_t *bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)tm), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, uint64_t *bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)tm), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// Slot of slice t in a K block of parity P.  Slice i of a block is last read
// at step max(i, S-1-i) (steps follow the slices as they arrive), so in odd
// blocks the first-needed slices go to the slots that the even block frees
// first, and the loads of a block overlap the last steps of the one before.
template <int S>
__host__ __device__ constexpr int release_step(int i) { return i > S - 1 - i ? i : S - 1 - i; }

template <int S>
__host__ __device__ constexpr int slot_of(int P, int t) {
    if (P == 0) return t;
    // the slot whose release rank (release step, then index) is t
    for (int i = 0; i < S; ++i) {
        int r = 0;
        for (int j = 0; j < S; ++j)
            r += (release_step<S>(j) < release_step<S>(i)) || (release_step<S>(j) == release_step<S>(i) && j < i);
        if (r == t) return i;
    }
    return 0;
}

// double-float accumulation: (hi, lo) += x, exact TwoSum on the high part
__device__ __forceinline__ void df_add(float &hi, float &lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// One K block of MMAs, fully unrolled for slot parity P: for each arriving
// slice t, the pairs (i, l) with max(i, l) = t and i + l < S, then the commits
// that free the slots read for the last time.
template <int S, int P>
__device__ __forceinline__ bool mma_block(uint64_t *full_bar, uint64_t *empty_bar, uint32_t par, uint32_t tmem,
                                          uint64_t desc0, uint32_t idesc, uint32_t &fresh, int *err) {
#pragma unroll
    for (int t = 0; t < S; ++t) {
        if (!mbar_wait(&full_bar[slot_of<S>(P, t)], par, err, 4)) return false;
        tc_fence_after();
#pragma unroll
        for (int i = 0; i <= t; ++i) {
#pragma unroll
            for (int l = 0; l <= t; ++l) {
                if ((i == t || l == t) && i + l < S) {
                    const int s = i + l < 3 ? i + l : 3;
                    const uint32_t offA = (uint32_t)(slot_of<S>(P, i) * SLOT);
                    const uint32_t offB = (uint32_t)(slot_of<S>(P, l) * SLOT + A_TILE);
#pragma unroll
                    for (int k = 0; k < BKB / 16; ++k) {
                        const uint32_t acc = (fresh >> s) & 1u ? 0u : 1u;
                        mma_bf16(tmem + s * BN, desc0 + ((offA + k * 32) >> 4), desc0 + ((offB + k * 32) >> 4), idesc,
                                 acc);
                        fresh &= ~(1u << s);
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < S; ++i)
            if (release_step<S>(i) == t) mma_commit(&empty_bar[slot_of<S>(P, i)]);
    }
    return true;
}

// Slot of slice t in stage G: slot set G mod NSET, or with a single set the
// release-ordered slots of odd stages.
template <int S, int NSET>
__device__ __forceinline__ int xslot_index(int G, int t) {
    if (NSET >= 2) return (G % NSET) * S + t;
    return (G & 1) ? slot_of<S>(1, t) : t;
}

// One K stage of the expansion kernel (stage G, slots xslot_index), with
// accumulators at TMEM column tacc: for each arriving slice t the pairs (i, l)
// with max(i, l) = t and i + l < S, then the commits that free the slots read
// for the last time.
template <int S, int TBN, int KS, int NSET>
__device__ __forceinline__ bool mma_stage(uint64_t *full_bar, uint64_t *empty_bar, int G, uint32_t tacc,
                                          uint64_t desc0, uint32_t idesc, uint32_t &fresh, int *err) {
    constexpr int XS = xslot(TBN, KS);
    const uint32_t par = (uint32_t)((G / NSET) & 1);
#pragma unroll
    for (int t = 0; t < S; ++t) {
        if (!mbar_wait(&full_bar[xslot_index<S, NSET>(G, t)], par, err, 4)) return false;
        tc_fence_after();
#pragma unroll
        for (int i = 0; i <= t; ++i) {
#pragma unroll
            for (int l = 0; l <= t; ++l) {
                if ((i == t || l == t) && i + l < S) {
                    const int s = i + l < 3 ? i + l : 3;
                    const uint32_t offA = (uint32_t)(xslot_index<S, NSET>(G, i) * XS);
                    const uint32_t offB = (uint32_t)(xslot_index<S, NSET>(G, l) * XS + xa_tile(KS));
#pragma unroll
                    for (int k = 0; k < KS / 16; ++k) {
                        const uint32_t acc = (fresh >> s) & 1u ? 0u : 1u;
                        mma_bf16(tacc + s * TBN, desc0 + ((offA + k * 32) >> 4), desc0 + ((offB + k * 32) >> 4),
                                 idesc, acc);
                        fresh &= ~(1u << s);
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < S; ++i)
            if (release_step<S>(i) == t) mma_commit(&empty_bar[xslot_index<S, NSET>(G, i)]);
    }
    return true;
}

// Fold one chunk's accumulators (NC columns of this thread's TMEM lane,
// accumulator s at column offset s * stride) into the double-float sums:
// s = 0, 1, 2 by TwoSum (2^-14 of the result for s = 2 still needs it to keep
// the low word below an ulp of the high one), s >= 3 (2^-21) into the low word.
template <int S, int NC>
__device__ __forceinline__ void drain_chunk(uint32_t tbase, int stride, float (&hi)[NC], float (&lo)[NC]) {
    constexpr int n_acc = S < 4 ? S : 4;       // accumulators written by the MMAs
    static_assert(NC % 16 == 0, "columns are loaded 16 at a time");
#pragma unroll
    for (int c0 = 0; c0 < NC; c0 += 16) {
        // two accumulators' 16 columns in flight together, one wait each pair
        uint32_t v[16], w[16];
        tmem_ld16_async(tbase + c0, v);
        if (n_acc > 1) tmem_ld16_async(tbase + stride + c0, w);
        tmem_wait_ld();
        tmem_regs_ready(v);
        if (n_acc > 1) tmem_regs_ready(w);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            df_add(hi[c0 + i], lo[c0 + i], __uint_as_float(v[i]));
            if (n_acc > 1) df_add(hi[c0 + i], lo[c0 + i], __uint_as_float(w[i]));
        }
        if (n_acc > 2) {
            tmem_ld16_async(tbase + 2 * stride + c0, v);
            if (n_acc > 3) tmem_ld16_async(tbase + 3 * stride + c0, w);
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

// Position of tile `tile` of a grouped launch: its task, the first rows of
// its continuum-pair block and its first column.
struct TilePos {
    int ti, jj0, jjp0, n0;
};

template <int TBN>
__device__ __forceinline__ TilePos tile_pos(const SplitTask *__restrict__ tasks, const int64_t *__restrict__ blk,
                                            int n_tasks, int tile) {
    TilePos p;
    p.ti = task_of(blk, n_tasks, tile);
    const int lb = (int)(tile - __ldg(blk + p.ti));
    const SplitTask &a = tasks[p.ti];
    const int ntn = a.ntn, jpt_tiles = a.jpt_tiles, lg = a.bjp_log2;
    const int tile_n = lb % ntn, tile_m = lb / ntn;   // N fastest: CTAs sharing a panel tile run together
    p.jj0 = (tile_m / jpt_tiles) * (BM >> lg);        // tile of (128 >> lg) j x (1 << lg) j'
    p.jjp0 = (tile_m % jpt_tiles) << lg;
    p.n0 = tile_n * TBN;
    return p;
}

// Persistent: each CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// The slot ring, the accumulator hand-over and their barrier phases run on
// across tiles, so the loads and MMAs of the next tile start while the
// epilogue warps still write the last one out from registers.
template <int S, int TBN, int KS>
__global__ void __launch_bounds__(NTHREADS, 1)
split_expand_kernel(const __grid_constant__ CUtensorMap tm_panel, const __grid_constant__ CUtensorMap tm_coef,
                    const SplitTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks, int n_tiles,
                    int kblocks, int coef_planes, const ExpCol *__restrict__ cols, int *err, int shard_r,
                    int shard_n) {
    // this launch's tiles: shard_r, shard_r + shard_n, ... (all of them unless
    // sharded), numbered t = 0, 1, ... so that every role walks the same list
    const int n_local = n_tiles > shard_r ? (n_tiles - shard_r + shard_n - 1) / shard_n : 0;
    constexpr int XS = xslot(TBN, KS);
    constexpr int NSET = xsets(S, TBN, KS);
    constexpr int NACC = xacc_bufs(TBN);      // accumulator sets in tensor memory
    constexpr int TCOLS = xtmem_cols(TBN);
    constexpr int ECOLS = TBN / 2;            // columns per epilogue thread
    constexpr int SPC = KCHUNK / KS;          // stages per exact chunk
    static_assert(KS == 32 || KS == 64, "stage width");
    static_assert(NSET >= 1 && NSET * S <= XBARS, "slot sets");
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *slots = base;                                         // [NSET][S][XS]
    uint64_t *full_bar = (uint64_t *)(base + NSET * S * XS);      // [XBARS]
    uint64_t *empty_bar = full_bar + XBARS;                        // [XBARS]
    uint64_t *acc_full = empty_bar + XBARS;                        // [2]
    uint64_t *acc_empty = acc_full + 2;                            // [2]
    uint64_t *final_bar = acc_empty + 2;                           // [1]
    uint32_t *tmem_slot = (uint32_t *)(final_bar + 1);
    // the epilogue's tile: arguments and column destinations, double-buffered
    __shared__ SplitTask ta[2];
    __shared__ TilePos tp[2];
    __shared__ ExpCol colmeta[2][TBN];
    __shared__ int epi_fail;                 // an epilogue wait gave up (read only after a barrier)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nst = kblocks * (64 / KS);     // K stages per tile
    const int nchunks = (nst + SPC - 1) / SPC;

    if (threadIdx.x == 0) {
        epi_fail = 0;
        for (int i = 0; i < XBARS; ++i) { mbar_init(&full_bar[i], 1); mbar_init(&empty_bar[i], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], EPI_THREADS); }
        mbar_init(final_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        if (lane == 0) {
            int G = 0;                            // K stages issued by this CTA over all its tiles
            bool ok = true;
            for (int t = blockIdx.x; t < n_local && ok; t += gridDim.x) {
                const int tile = shard_r + shard_n * t;
                const TilePos p = tile_pos<TBN>(tasks, blk, n_tasks, tile);
                const int cx = tasks[p.ti].cfp + p.jjp0, cy = tasks[p.ti].cf + p.jj0;
                const int crow = (int)(tasks[p.ti].coef_row0 + p.n0);
                const int kc0 = tasks[p.ti].kc0;      // the block's label class in the coefficient slices
                for (int ks = 0; ks < nst && ok; ++ks, ++G) {
                    // stage G uses its slots for the (G / NSET)-th time
                    const int round = G / NSET;
                    const int kx = KS == 64 ? 0 : (ks & 1) * 32;   // part of 64-wide K block kb
                    const int kb = KS == 64 ? ks : ks >> 1;
                    for (int t = 0; t < S && ok; ++t) {
                        const int sl = xslot_index<S, NSET>(G, t);
                        // wait for the slot's release by the stage NSET before this one
                        if (round > 0) ok = mbar_wait(&empty_bar[sl], (round - 1) & 1, err, 1);
                        if (!ok) break;
                        uint8_t *sA = slots + sl * XS;
                        mbar_expect_tx(&full_bar[sl], (uint32_t)XS);
                        tma_load_4d(sA, &tm_panel, &full_bar[sl], kx, cx, cy, t * kblocks + kb);
                        tma_load_3d(sA + xa_tile(KS), &tm_coef, &full_bar[sl], kx, crow,
                                    t * coef_planes + kc0 + kb);
                    }
                }
            }
            // wait until this producer's copies of the last stage of every set have landed
            for (int g = G > NSET ? G - NSET : 0; g < G; ++g)
                for (int t = 0; t < S; ++t)
                    mbar_wait(&full_bar[xslot_index<S, NSET>(g, t)], (g / NSET) & 1, err, 2);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = instr_desc_bf16(BM, TBN);
            // + (offset >> 4) per operand tile
            const uint64_t desc0 = KS == 64 ? smem_desc_sw128(smem_u32(slots)) : smem_desc_sw64(smem_u32(slots));
            bool ok = true;
            int G = 0, C = 0;                     // K stages and chunks over all tiles
            for (int t = blockIdx.x; t < n_local && ok; t += gridDim.x) {
                for (int c = 0; c < nchunks && ok; ++c, ++C) {
                    // chunk C fills accumulator set C mod NACC, drained after chunk C - NACC
                    const int b = C % NACC;
                    if (C >= NACC) ok = mbar_wait(&acc_empty[b], (C / NACC - 1) & 1, err, 3);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t tacc = tmem + (uint32_t)(b * 4 * TBN);
                    const int ks_end = min(nst, (c + 1) * SPC);
                    uint32_t fresh = 0xFu;        // accumulators not yet written in this chunk
                    for (int ks = c * SPC; ks < ks_end && ok; ++ks, ++G)
                        ok = mma_stage<S, TBN, KS, NSET>(full_bar, empty_bar, G, tacc, desc0, idesc, fresh, err);
                    if (ok) mma_commit(&acc_full[b]);     // accumulators of chunk C complete
                }
            }
            mma_commit(final_bar);
            mbar_wait(final_bar, 0, err, 5);
        }
    } else {
        // ------------------------------------------------------ epilogue
        const int e = threadIdx.x - 64;          // 0 .. EPI_THREADS-1
        const int ew = warp - 2;
        const int q = warp & 3;                  // TMEM lane quadrant this warp may access
        const int col0 = (ew >> 2) * ECOLS;
        const int row = q * 32 + lane;           // tile row = TMEM lane
        int C = 0, it = 0;
        for (int t = blockIdx.x; t < n_local; t += gridDim.x, ++it) {
            const int tile = shard_r + shard_n * t;
            const int buf = it & 1;
            // the buffer was last read by the stores of tile it-2, which every
            // epilogue warp finished before the barriers of tile it-1
            if (e == 0) {
                tp[buf] = tile_pos<TBN>(tasks, blk, n_tasks, tile);
                ta[buf] = tasks[tp[buf].ti];
            }
            // every epilogue thread reaches both barriers of a tile, so the
            // failure flag read after the first is the same for all of them
            named_bar_sync(1, EPI_THREADS);
            if (epi_fail) break;
            const SplitTask &a = ta[buf];
            if (e < TBN) {
                const int t = tp[buf].n0 + e;
                ExpCol cm;
                if (t < a.N) cm = cols[a.col0 + t];
                else cm.H = nullptr;
                colmeta[buf][e] = cm;
            }
            named_bar_sync(1, EPI_THREADS);
            float hi[ECOLS], lo[ECOLS];
#pragma unroll
            for (int c = 0; c < ECOLS; ++c) { hi[c] = 0.0f; lo[c] = 0.0f; }
            bool ok = true;
            for (int c = 0; c < nchunks; ++c, ++C) {
                const int b = C % NACC;
                if (ok) ok = mbar_wait(&acc_full[b], (C / NACC) & 1, err, 6);
                if (!ok) continue;
                tc_fence_after();
                drain_chunk<S>(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 4 * TBN + col0), TBN, hi, lo);
                tc_fence_before();
                mbar_arrive(&acc_empty[b]);
            }
            if (!ok) {
                epi_fail = 1;
                continue;                        // leaves at the next tile's first barrier
            }
            // the accumulators are free again: the MMAs of the next tile run
            // while this one is written out
            const int lg = a.bjp_log2;
            const int jj = tp[buf].jj0 + (row >> lg), jjp = tp[buf].jjp0 + (row & ((1 << lg) - 1));
            if (jj < a.cn && jjp < a.cnp && (a.cf + jj) != (a.cfp + jjp)) {
#pragma unroll
                for (int c = 0; c < ECOLS; ++c) {
                    const ExpCol &m = colmeta[buf][col0 + c];
                    if (m.H) {
                        const int64_t r = m.rbase + jj;
                        const int64_t cc = m.cbase + jjp;
                        if (!m.same || r >= cc) {
                            const double v = df_to_double(hi[c], lo[c]);
                            m.H[r * m.ld + cc] = v;
                            if (r != cc) m.H[cc * m.ld + r] = v;
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS) : "memory");
    }
}

// ------------------------------------------- dense split GEMM (Davidson)
// part[z][n][m] = sum over the K blocks of split z of A[m][k] X[n][k], for the
// Davidson block products H V: A (rows m of the Hamiltonian) and X (rows n =
// the block's vectors) as bf16 slices with their row exponents folded in,
// the same exact slice-pair accumulation as the expansion kernel; the K
// dimension is split over blockIdx.z (one exact chunk each) and the
// double-float partials are summed in a fixed order by dense_reduce_kernel.
struct DenseArgs {
    int M, N;                  // rows of A and of X
    int kb_total, kb_per_split;
    int a_planes, b_planes;    // K blocks per slice plane of A and of X
    float2 *part;              // [nsplit][N][M]
    int *err;
};

template <int S>
__global__ void __launch_bounds__(NTHREADS, 1)
dense_split_kernel(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b, DenseArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *slots = base;
    uint64_t *full_bar = (uint64_t *)(base + S * SLOT);
    uint64_t *empty_bar = full_bar + MAXS;
    uint64_t *acc_full = empty_bar + MAXS;
    uint64_t *acc_empty = acc_full + 1;
    uint64_t *final_bar = acc_empty + 1;
    uint32_t *tmem_slot = (uint32_t *)(final_bar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM, z = blockIdx.z;
    const int kb0 = z * a.kb_per_split;
    const int kb1 = min(a.kb_total, kb0 + a.kb_per_split);
    const int nkb = kb1 - kb0;
    const int kb_per_chunk = KCHUNK / BKB;
    const int nchunks = (nkb + kb_per_chunk - 1) / kb_per_chunk;
    int *err = a.err;
    if (threadIdx.x == 0) {
        for (int i = 0; i < MAXS; ++i) { mbar_init(&full_bar[i], 1); mbar_init(&empty_bar[i], 1); }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, EPI_THREADS);
        mbar_init(final_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (warp == 0) {
        // TMA producer (kk: K block within this split, for slot parity and phases)
        if (lane == 0) {
            int kk = 0;
            bool ok = true;
            for (; kk < nkb && ok; ++kk) {
                const int kb = kb0 + kk;
                for (int t = 0; t < S && ok; ++t) {
                    const int sl = (kk & 1) ? slot_of<S>(1, t) : t;
                    if (kk > 0) ok = mbar_wait(&empty_bar[sl], (kk - 1) & 1, err, 1);
                    if (!ok) break;
                    uint8_t *sA = slots + sl * SLOT;
                    mbar_expect_tx(&full_bar[sl], (uint32_t)SLOT);
                    tma_load_3d(sA, &tm_a, &full_bar[sl], 0, m0, t * a.a_planes + kb);
                    tma_load_3d(sA + A_TILE, &tm_b, &full_bar[sl], 0, n0, t * a.b_planes + kb);
                }
            }
            if (kk > 0)
                for (int sl = 0; sl < S; ++sl) mbar_wait(&full_bar[sl], (kk - 1) & 1, err, 2);
        }
    } else if (warp == 1) {
        // MMA issuer
        if (lane == 0) {
            const uint32_t idesc = instr_desc_bf16(BM, BN);
            const uint64_t desc0 = smem_desc_sw128(smem_u32(slots));
            bool ok = true;
            int kk = 0;
            for (int c = 0; c < nchunks && ok; ++c) {
                if (c > 0) ok = mbar_wait(acc_empty, (c - 1) & 1, err, 3);
                if (!ok) break;
                tc_fence_after();
                const int kk_end = min(nkb, (c + 1) * kb_per_chunk);
                uint32_t fresh = 0xFu;
                for (; kk < kk_end && ok; ++kk) {
                    if (kk & 1) ok = mma_block<S, 1>(full_bar, empty_bar, 1u, tmem, desc0, idesc, fresh, err);
                    else ok = mma_block<S, 0>(full_bar, empty_bar, 0u, tmem, desc0, idesc, fresh, err);
                }
                if (ok) mma_commit(acc_full);
            }
            mma_commit(final_bar);
            mbar_wait(final_bar, 0, err, 5);
        }
    } else {
        // epilogue: rows m of A = TMEM lanes, columns = vectors n
        const int ew = warp - 2;
        const int q = warp & 3;
        const int col0 = (ew >> 2) * EPI_COLS;
        const int row = q * 32 + lane;
        float hi[EPI_COLS], lo[EPI_COLS];
#pragma unroll
        for (int c = 0; c < EPI_COLS; ++c) { hi[c] = 0.0f; lo[c] = 0.0f; }
        bool ok = true;
        for (int c = 0; c < nchunks && ok; ++c) {
            ok = mbar_wait(acc_full, c & 1, err, 6);
            if (!ok) break;
            tc_fence_after();
            drain_chunk<S>(tmem + ((uint32_t)(q * 32) << 16) + col0, BN, hi, lo);
            tc_fence_before();
            mbar_arrive(acc_empty);
        }
        const int m = m0 + row;
        if (ok && m < a.M) {
            float2 *out = a.part + (int64_t)z * a.N * a.M + m;
#pragma unroll
            for (int c = 0; c < EPI_COLS; ++c) {
                const int n = n0 + col0 + c;
                if (n < a.N) out[(int64_t)n * a.M] = make_float2(hi[c], lo[c]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Y[n][m] (row stride ldy) = sum over the splits, in order, of part[z][n][m].
__global__ void dense_reduce_kernel(const float2 *__restrict__ part, int nsplit, int M, int N, double *__restrict__ Y,
                                    int64_t ldy) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)M * N) return;
    const int n = (int)(t / M), m = (int)(t % M);
    float h = 0.0f, l = 0.0f;
    for (int z = 0; z < nsplit; ++z) {
        const float2 x = part[((int64_t)z * N + n) * M + m];
        df_add2(h, l, x.x, x.y);
    }
    Y[(int64_t)n * ldy + m] = df_to_double(h, l);
}

// One row into its S bf16 slices by a whole block (the digits of slice_row):
// every thread reads its share of the row, the row exponent is reduced through
// shared memory, then each thread writes the digits of its elements.  at(k)
// gives element k (0 beyond the row's data).
template <class At>
__device__ __forceinline__ void slice_row_block(At at, int64_t dest, int64_t R, int Kpad, int S,
                                                __nv_bfloat16 *__restrict__ out) {
    __shared__ int red[32];
    int emax = -2000;
    for (int k = threadIdx.x; k < Kpad; k += blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(at(k));
        const int be = (int)((b >> 52) & 0x7FF);
        if (be == 0) continue;                 // zero (FP64 subnormals ignored)
        const int e = be - 1022;               // |x| in [2^(e-1), 2^e)
        emax = e > emax ? e : emax;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const int o = __shfl_xor_sync(0xffffffffu, emax, off);
        emax = o > emax ? o : emax;
    }
    const int warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) red[warp] = emax;
    __syncthreads();
    emax = -2000;
    for (int w = 0; w < nw; ++w) emax = red[w] > emax ? red[w] : emax;
    const int KB = Kpad / BKB;
    for (int k = threadIdx.x; k < Kpad; k += blockDim.x) {
        long long F = 0;
        if (emax > -2000) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(at(k));
            const int be = (int)((b >> 52) & 0x7FF);
            if (be != 0) {
                const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));   // x = m 2^(be-1075)
                const int sh = (be - 1075) + 7 * S - emax;      // F = m 2^sh, rounded to nearest
                long long f;
                if (sh >= 0) f = m << sh;
                else if (sh > -63) f = (m + (1ll << (-sh - 1))) >> (-sh);
                else f = 0;
                F = (b >> 63) ? -f : f;
            }
        }
        const int kb = k / BKB, kk = k % BKB;
        for (int i = 0; i < S; ++i) {
            const int sh = 7 * (S - 1 - i);
            long long d = sh > 0 ? ((F + (1ll << (sh - 1))) >> sh) : F;   // nearest digit
            F -= d << sh;
            out[(((int64_t)i * KB + kb) * R + dest) * BKB + kk] =
                __float2bfloat16_rn(ldexpf((float)d, emax - 7 - 7 * i));   // exact: |d| <= 128
        }
    }
}

// Rows of [X1 | X2] (K1 then K2 entries, row strides ld1, ld2; X2 may be
// absent) into bf16 slices [S][Kpad/64][R][64], one block per row.
__global__ void __launch_bounds__(1024)
slice_rows2_kernel(const double *__restrict__ X1, int64_t ld1, int K1, const double *__restrict__ X2, int64_t ld2,
                   int K2, int Kpad, int S, int64_t R, __nv_bfloat16 *__restrict__ out) {
    const int64_t row = blockIdx.x;
    const double *x1 = X1 + row * ld1;
    const double *x2 = X2 ? X2 + row * ld2 : nullptr;
    slice_row_block([&](int k) -> double { return k < K1 ? __ldg(x1 + k) : ((x2 && k < K1 + K2) ? __ldg(x2 + k - K1) : 0.0); },
                    row, R, Kpad, S, out);
}

// ------------------------------------------------------------- slicing
// One warp per row.  Row maximum |x|, e with max < 2^e; each element becomes
// the 64-bit fixed-point integer F = round(x 2^{7S-e}) (|F| < 2^{7S}, built
// from the FP64 bit pattern with integer operations), whose balanced base-128
// digits d_0 .. d_{S-1} (d_0 in [-128, 128], the rest in [-64, 64]) are the
// slices: slice i = d_i 2^{e-7-7i}.  Output layout [S][K/64][R][64] (R rows in
// all), so a 64-wide K block of consecutive rows is contiguous.  Column
// skip_col is zero.
__device__ __forceinline__ void slice_row(const double *__restrict__ x, int64_t dest, int64_t R, int Kpad, int S,
                                          int skip_col, __nv_bfloat16 *__restrict__ out, int lane) {
    const int KB = Kpad / BKB;
    // exponent of the row maximum from the bit patterns (no FP64 arithmetic)
    int emax = -2000;
    for (int k = lane; k < Kpad; k += 32) {
        if (k == skip_col) continue;
        const unsigned long long b = (unsigned long long)__double_as_longlong(x[k]);
        const int be = (int)((b >> 52) & 0x7FF);
        if (be == 0) continue;                 // zero (FP64 subnormals ignored)
        const int e = be - 1022;               // |x| in [2^(e-1), 2^e)
        emax = e > emax ? e : emax;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const int o = __shfl_xor_sync(0xffffffffu, emax, off);
        emax = o > emax ? o : emax;
    }
    for (int k = lane; k < Kpad; k += 32) {
        long long F = 0;
        if (k != skip_col && emax > -2000) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(x[k]);
            const int be = (int)((b >> 52) & 0x7FF);
            if (be != 0) {
                const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));   // x = m 2^(be-1075)
                const int sh = (be - 1075) + 7 * S - emax;      // F = m 2^sh, rounded to nearest
                long long f;
                if (sh >= 0) f = m << sh;                       // sh <= 7S - 53 < 0 in practice
                else if (sh > -63) f = (m + (1ll << (-sh - 1))) >> (-sh);
                else f = 0;
                F = (b >> 63) ? -f : f;
            }
        }
        const int kb = k / BKB, kk = k % BKB;
        for (int i = 0; i < S; ++i) {
            const int sh = 7 * (S - 1 - i);
            long long d = sh > 0 ? ((F + (1ll << (sh - 1))) >> sh) : F;   // nearest digit (floor of F/2^sh + 1/2)
            F -= d << sh;
            const float v = ldexpf((float)d, emax - 7 - 7 * i);            // exact: |d| <= 128
            out[(((int64_t)i * KB + kb) * R + dest) * BKB + kk] = __float2bfloat16_rn(v);
        }
    }
}

// Panel rows (j n_co + j') into slices; column skip_col (the delta label) is
// zeroed on the rows with j == j' (elsewhere that label is zero, or, with
// orbital symmetry, the column holds another label).
__global__ void slice_rows_kernel(const double *__restrict__ X, int64_t rows, int Kpad, int S, int skip_col,
                                  int n_co, __nv_bfloat16 *__restrict__ out) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    const bool diag = row / n_co == row % n_co;
    slice_row(X + row * Kpad, row, rows, Kpad, S, diag ? skip_col : -1, out, threadIdx.x & 31);
}

// Coefficient rows (Kin entries each) into slices of Kout columns: column k
// holds label perm[k] (the labels class by class, with orbital symmetry; -1
// padding), or label k without a permutation; column skip_col (the delta
// label) is zero.
__global__ void __launch_bounds__(256)
slice_rows_grouped(const SliceTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks, int64_t R,
                   int Kin, int Kout, const int32_t *__restrict__ perm, int S, int skip_col,
                   __nv_bfloat16 *__restrict__ out) {
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const SliceTask &T = tasks[ti];
    const int64_t row = blockIdx.x - blk[ti];
    const double *x = T.X + row * Kin;
    slice_row_block([&](int k) -> double {
        if (k == skip_col) return 0.0;
        const int lab = perm ? __ldg(perm + k) : k;
        return (lab >= 0 && lab < Kin) ? __ldg(x + lab) : 0.0;
    }, T.row0 + row, R, Kout, S, out);
}

// Rows with j == j' (both ranges): H[(n,j),(n',j)] over all K, incl. delta,
// in double-float (they carry h_jj and the delta_jj' E term and so have a
// wide dynamic range that the bf16 slices of one row do not cover).  Per task
// one block per (j, 8 state pairs); the lanes of a warp split K.
// A block computes a tile of kDRj rows j x kDRt coefficient rows t; the
// panel and coefficient rows pass through shared memory in K-chunks (the next
// chunk is read into registers while the current one is used) and every
// thread keeps four double-float partial sums (k mod 4), combined in a fixed
// order at the end.
constexpr int kDRj = 16, kDRt = 16, kDRk = 128;
constexpr int kDRthreads = kDRj * kDRt;
constexpr int kDRper = kDRj * kDRk / kDRthreads;     // elements of each tile a thread moves per chunk

__global__ void __launch_bounds__(kDRthreads)
diag_rows_kernel(const DRTask *__restrict__ tasks, const int64_t *__restrict__ blk, int n_tasks) {
    static_assert(kDRj == kDRt, "both tiles are moved by the same index pattern");
    __shared__ float2 sp[kDRj][kDRk + 1], sa[kDRt][kDRk + 1];
    const int ti = task_of(blk, n_tasks, blockIdx.x);
    const DRTask &T = tasks[ti];
    const int lb = (int)(blockIdx.x - blk[ti]);
    const int j0 = T.j_lo + (lb / T.ny) * kDRj, t0 = (lb % T.ny) * kDRt;
    const int tl = threadIdx.x % kDRt, jl = threadIdx.x / kDRt;
    const int j = j0 + jl, t = t0 + tl;
    const int Kpad = T.Kpad, Ka = T.Ka, j_hi = T.j_hi, n_nn = T.n_nn;
    const float2 *__restrict__ Pd = T.Pd;
    const float2 *__restrict__ A = T.A;
    const int32_t *__restrict__ perm = T.perm;
    float2 rp[kDRper], ra[kDRper];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int u = 0; u < kDRper; ++u) {
            const int i = threadIdx.x + u * kDRthreads;
            const int r = i / kDRk, k = k0 + i % kDRk;
            const bool kin = k < Kpad;
            rp[u] = (kin && j0 + r < j_hi) ? __ldg(Pd + (int64_t)(j0 + r) * Kpad + k) : make_float2(0.0f, 0.0f);
            const int lab = (kin && perm) ? __ldg(perm + k) : k;   // the label of panel column k
            ra[u] = (kin && lab >= 0 && t0 + r < n_nn) ? __ldg(A + (int64_t)(t0 + r) * Ka + lab)
                                                        : make_float2(0.0f, 0.0f);
        }
    };
    float h[4] = {0.0f, 0.0f, 0.0f, 0.0f}, l[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    fetch(0);
    for (int k0 = 0; k0 < Kpad; k0 += kDRk) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kDRper; ++u) {
            const int i = threadIdx.x + u * kDRthreads;
            sp[i / kDRk][i % kDRk] = rp[u];
            sa[i / kDRk][i % kDRk] = ra[u];
        }
        __syncthreads();
        if (k0 + kDRk < Kpad) fetch(k0 + kDRk);
#pragma unroll 2
        for (int k = 0; k < kDRk; k += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 x = sp[jl][k + u], y = sa[tl][k + u];
                df_fma(h[u], l[u], x.x, x.y, y.x, y.y);
            }
        }
    }
    if (j >= j_hi || t >= n_nn) return;
    df_add2(h[0], l[0], h[1], l[1]);
    df_add2(h[2], l[2], h[3], l[3]);
    df_add2(h[0], l[0], h[2], l[2]);
    const int na = T.nn[2 * t], nb = T.nn[2 * t + 1];
    const int64_t r = T.row_off + (int64_t)na * T.cn + (j - T.cf);
    const int64_t c = T.col_off + (int64_t)nb * T.cnp + (j - T.cfp);
    if (T.same && r < c) return;
    const double v = df_to_double(h[0], l[0]);
    T.H[r * T.ld + c] = v;
    if (r != c) T.H[c * T.ld + r] = v;
}

// Diagonal panel rows P[(j, j)][k] as float pairs.
__global__ void panel_diag_df_kernel(const double *__restrict__ P, int n_co, int Kpad, float2 *__restrict__ out) {
    const int j = blockIdx.x;
    for (int k = threadIdx.x; k < Kpad; k += blockDim.x) {
        const double v = P[((int64_t)j * n_co + j) * Kpad + k];
        const float h = (float)v;
        out[(int64_t)j * Kpad + k] = make_float2(h, (float)(v - (double)h));
    }
}

// ------------------------------------------------------ tensor maps (host)
typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
    });
    return fn;
}

}  // namespace

// dynamic shared memory of the expansion kernel: the operand slots, the
// barriers and the 1 KB alignment
static int split_smem_bytes(int S, int bn, int ks) { return xsets(S, bn, ks) * S * xslot(bn, ks) + 2048; }

static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 1;
    }
    return n;
}

template <int S>
static cudaError_t set_smem_attr_s() {
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(split_expand_kernel<S, 32, 32>, attr, split_smem_bytes(S, 32, 32));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(split_expand_kernel<S, 64, 32>, attr, split_smem_bytes(S, 64, 32));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(split_expand_kernel<S, 128, 32>, attr, split_smem_bytes(S, 128, 32));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(split_expand_kernel<S, 128, 64>, attr, split_smem_bytes(S, 128, 64));
    return e;
}

static cudaError_t set_smem_attr(int S) {
    switch (S) {
        case 2: return set_smem_attr_s<2>();
        case 3: return set_smem_attr_s<3>();
        case 4: return set_smem_attr_s<4>();
        case 5: return set_smem_attr_s<5>();
        default: return set_smem_attr_s<6>();
    }
}

static int mixed_fail(hb_ctx *ctx, int code, const std::string &m) {
    ctx->err = m;
    return code;
}

// Panel slices and their tensor map, once per context (the integrals do not
// change between builds); a context that borrows its integrals borrows these.
int mixed_prepare(hb_ctx *ctx, cudaStream_t s) {
    if (!ctx->mixed) ctx->mixed = new MixedState();
    MixedState &M = *ctx->mixed;
    if (M.panel_ready) return HB_OK;
    if (ctx->base) {
        int rc = mixed_prepare(ctx->base, s);
        if (rc != HB_OK) return mixed_fail(ctx, rc, ctx->base->err);
        const MixedState &B = *ctx->base->mixed;
        M.slices = B.slices;
        M.panel_rows = B.panel_rows;
        M.panel_slices = B.panel_slices;
        for (int w = 0; w < 2; ++w)
            for (int i = 0; i < 3; ++i) M.tm_panel[w][i] = B.tm_panel[w][i];
        M.pdiag = B.pdiag;
        M.borrowed_panel = true;
        M.panel_ready = true;
        return HB_OK;
    }
    M.slices = ctx->split_slices;
    if (M.slices < 2 || M.slices > MAXS) return mixed_fail(ctx, HB_ERR_INVALID_ARG, "split_slices must be 2..6");
    if (!encode_fn()) return mixed_fail(ctx, HB_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    const int64_t rows = (int64_t)ctx->n_co * ctx->n_co;
    M.panel_rows = rows;
    // the panel's columns: every label, or with orbital symmetry the Kc labels
    // of each row's class
    const int Kc = ctx->Kc;
    cudaError_t e = dmalloc(ctx, (void **)&M.panel_slices, sizeof(__nv_bfloat16) * (size_t)M.slices * rows * Kc);
    if (e != cudaSuccess) return mixed_fail(ctx, HB_ERR_OOM, std::string("panel slices: ") + cudaGetErrorString(e));
    ctx->dev_bytes += sizeof(__nv_bfloat16) * (size_t)M.slices * rows * Kc;
    e = dmalloc_n(ctx, &M.pdiag, (size_t)ctx->n_co * Kc);
    if (e != cudaSuccess) return mixed_fail(ctx, HB_ERR_OOM, std::string("panel rows: ") + cudaGetErrorString(e));
    ctx->dev_bytes += sizeof(float2) * (size_t)ctx->n_co * Kc;
    panel_diag_df_kernel<<<ctx->n_co, 256, 0, s>>>(ctx->panel, ctx->n_co, Kc, M.pdiag);
    slice_rows_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(ctx->panel, rows, Kc, M.slices, ctx->delta_pos,
                                                                 ctx->n_co, M.panel_slices);
    // 4D map over the panel slices [S*KB][j][j'][64]: coordinates (kk, j', j, plane)
    const int KB = Kc / BKB;
    cuuint64_t dims[4] = {(cuuint64_t)BKB, (cuuint64_t)ctx->n_co, (cuuint64_t)ctx->n_co,
                          (cuuint64_t)M.slices * KB};
    cuuint64_t strides[3] = {(cuuint64_t)BKB * 2, (cuuint64_t)ctx->n_co * BKB * 2, (cuuint64_t)rows * BKB * 2};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = CUDA_SUCCESS;
    for (int w = 0; w < 2 && r == CUDA_SUCCESS; ++w)
        for (int i = 0; i < 3 && r == CUDA_SUCCESS; ++i) {
            const int lg = 3 + i;
            // a 32-K stage copies half a 64-wide K block (x = 0 or 32: 64-byte
            // aligned, 64-byte swizzle), a 64-K stage all of it (128-byte swizzle)
            cuuint32_t box[4] = {w ? 64u : 32u, (cuuint32_t)(1 << lg), (cuuint32_t)(BM >> lg), 1};
            r = encode_fn()(&M.tm_panel[w][i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, M.panel_slices, dims, strides,
                            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            w ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        }
    if (r != CUDA_SUCCESS) return mixed_fail(ctx, HB_ERR_CUDA, "panel tensor map: error " + std::to_string((int)r));
    e = set_smem_attr(M.slices);
    if (e != cudaSuccess) return mixed_fail(ctx, HB_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e));
    M.panel_ready = true;
    return HB_OK;
}

const void *mixed_panel_key(const hb_ctx *ctx) { return ctx->mixed ? ctx->mixed->panel_slices : nullptr; }
const float2 *mixed_panel_diag(const hb_ctx *ctx) { return ctx->mixed ? ctx->mixed->pdiag : nullptr; }
int mixed_slices(const hb_ctx *ctx) { return ctx->mixed ? ctx->mixed->slices : ctx->split_slices; }

// Coefficient slices of `rows` rows in all: [S][Kpad/64][rows][64] bf16 and
// four 3D maps: for 32-K stages one per tile width bn = 32, 64, 128 (box: bn
// rows x half a K block of one slice plane, 64-byte swizzle), and for 64-K
// stages one of 128 rows x a whole K block (128-byte swizzle).
int split_coef_alloc(hb_ctx *mem, int S, int64_t rows, int Kpad, void **buf, CUtensorMap *tm, std::string *err) {
    *buf = nullptr;
    if (!encode_fn()) { *err = "cuTensorMapEncodeTiled is not available"; return HB_ERR_CUDA; }
    if (rows < 1) rows = 1;
    cudaError_t e = dmalloc(mem, buf, sizeof(__nv_bfloat16) * (size_t)S * rows * Kpad);
    if (e != cudaSuccess) { *err = std::string("coefficient slices: ") + cudaGetErrorString(e); return HB_ERR_OOM; }
    const int KB = Kpad / BKB;
    cuuint64_t dims[3] = {(cuuint64_t)BKB, (cuuint64_t)rows, (cuuint64_t)S * KB};
    cuuint64_t strides[2] = {(cuuint64_t)BKB * 2, (cuuint64_t)rows * BKB * 2};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = CUDA_SUCCESS;
    for (int i = 0; i < 4 && r == CUDA_SUCCESS; ++i) {
        cuuint32_t box[3] = {i < 3 ? 32u : 64u, (cuuint32_t)(i < 3 ? 32 << i : 128), 1};
        r = encode_fn()(&tm[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, *buf, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, i < 3 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) {
        dfree(mem, *buf);
        *buf = nullptr;
        *err = "coefficient tensor map: error " + std::to_string((int)r);
        return HB_ERR_CUDA;
    }
    return HB_OK;
}

int64_t blocks_split(int cn, int cnp, int N, int lg, int bn) {
    if (cn <= 0 || cnp <= 0 || N <= 0) return 0;
    const int bj = BM >> lg, bjp = 1 << lg;
    return (int64_t)((N + bn - 1) / bn) * ((cn + bj - 1) / bj) * ((cnp + bjp - 1) / bjp);
}
int split_ntn(int N, int bn) { return (N + bn - 1) / bn; }

// Tile width for a merged block of N columns over kblocks 64-wide K blocks:
// the narrowest of 32 and 64 that holds them, else 128 (whose MMAs read the
// least shared memory per flop).  Over long K every tile is 128 wide, so that
// every tile of the plan takes the same K stage (64) and a block's bits do not
// depend on the columns it is merged with.  `force` (32, 64, 128) overrides.
int split_cols_choice(int N, int kblocks, int force) {
    if (force == 32 || force == 64 || force == 128) return force;
    if (kblocks >= kK64Blocks) return 128;
    return N <= 32 ? 32 : (N <= 64 ? 64 : 128);
}
int split_jpt(int cnp, int lg) { return (cnp + (1 << lg) - 1) >> lg; }

// Tile arrangement with the least padding of the cn x cnp rectangle (ties: 8 x 16).
int split_tile_heuristic(int cn, int cnp) {
    int best = 4;
    int64_t best_area = -1;
    for (int lg : {4, 3, 5}) {
        const int bj = BM >> lg, bjp = 1 << lg;
        const int64_t area = (int64_t)((cn + bj - 1) / bj) * bj * ((cnp + bjp - 1) / bjp) * bjp;
        if (best_area < 0 || area < best_area) { best = lg; best_area = area; }
    }
    return best;
}

int g_slice(const Grouped<SliceTask> &g, int64_t R, int Kin, int Kout, const int32_t *perm, int S, int skip_col,
            void *out, cudaStream_t s) {
    if (g.blocks <= 0) return 0;
    slice_rows_grouped<<<(unsigned)g.blocks, 256, 0, s>>>(g.tasks, g.blk, g.n, R, Kin, Kout, perm, S, skip_col,
                                                          (__nv_bfloat16 *)out);
    return 1;
}

int split_kstage_choice(int bn, int kblocks, int force) {
    if (bn != 128) return 32;
    if (force == 32 || force == 64) return force;
    return kblocks >= kK64Blocks ? 64 : 32;
}

int g_split(const hb_ctx *panel_ctx, int lg, int bn, const CUtensorMap *tm_coef, const Grouped<SplitTask> &g,
            int kblocks, int coef_planes, const ExpCol *cols, int *err, cudaStream_t s, int shard_r, int shard_n) {
    if (g.blocks <= 0) return 0;
    if (bn != 32 && bn != 64 && bn != 128) return 0;
    const MixedState &M = *panel_ctx->mixed;
    const int ks = split_kstage_choice(bn, kblocks, panel_ctx->force_kstage);
    const CUtensorMap &tm_panel = M.tm_panel[ks == 64 ? 1 : 0][lg - 3];
    const CUtensorMap &tm_c = tm_coef[ks == 64 ? 3 : (bn == 32 ? 0 : (bn == 64 ? 1 : 2))];
    const size_t smem = split_smem_bytes(M.slices, bn, ks);
    // persistent: one CTA per SM at most (each holds its SM's tensor memory or half of it)
    const int n_tiles = (int)g.blocks;
    const int n_local = n_tiles > shard_r ? (n_tiles - shard_r + shard_n - 1) / shard_n : 0;
    if (n_local <= 0) return 0;
    const unsigned grid = (unsigned)std::min(n_local, sm_count());
#define HB_SPLIT(SS, BB, KK)                                                                                    \
    split_expand_kernel<SS, BB, KK><<<grid, NTHREADS, smem, s>>>(tm_panel, tm_c, g.tasks, g.blk, g.n, n_tiles, \
                                                                kblocks, coef_planes, cols, err, shard_r, shard_n)
#define HB_SPLIT_S(SS)                                 \
    do {                                               \
        if (bn == 32) HB_SPLIT(SS, 32, 32);            \
        else if (bn == 64) HB_SPLIT(SS, 64, 32);       \
        else if (ks == 32) HB_SPLIT(SS, 128, 32);      \
        else HB_SPLIT(SS, 128, 64);                    \
    } while (0)
    switch (M.slices) {
        case 2: HB_SPLIT_S(2); break;
        case 3: HB_SPLIT_S(3); break;
        case 4: HB_SPLIT_S(4); break;
        case 5: HB_SPLIT_S(5); break;
        default: HB_SPLIT_S(6); break;
    }
#undef HB_SPLIT_S
#undef HB_SPLIT
    return 1;
}

int64_t blocks_diag_rows(int j_lo, int j_hi, int n_nn) {
    if (j_hi <= j_lo || n_nn <= 0) return 0;
    return (int64_t)((j_hi - j_lo + kDRj - 1) / kDRj) * ((n_nn + kDRt - 1) / kDRt);
}
int diag_rows_ny(int n_nn) { return (n_nn + kDRt - 1) / kDRt; }

int g_diag_rows(const Grouped<DRTask> &g, cudaStream_t s) {
    if (g.blocks <= 0) return 0;
    diag_rows_kernel<<<(unsigned)g.blocks, kDRthreads, 0, s>>>(g.tasks, g.blk, g.n);
    return 1;
}

// ------------------------------------------------ dense split GEMM (host)
int dense_operand_alloc(hb_ctx *mem, int S, int64_t R, int Kpad, DenseOperand *op, std::string *err) {
    op->buf = nullptr;
    op->R = R < 1 ? 1 : R;
    op->Kpad = Kpad;
    op->planes = Kpad / BKB;
    if (!encode_fn()) { *err = "cuTensorMapEncodeTiled is not available"; return HB_ERR_CUDA; }
    const size_t bytes = sizeof(__nv_bfloat16) * (size_t)S * op->planes * op->R * BKB;
    cudaError_t e = dmalloc(mem, (void **)&op->buf, bytes);
    if (e != cudaSuccess) { *err = std::string("Davidson operand slices: ") + cudaGetErrorString(e); return HB_ERR_OOM; }
    cuuint64_t dims[3] = {(cuuint64_t)BKB, (cuuint64_t)op->R, (cuuint64_t)S * op->planes};
    cuuint64_t strides[2] = {(cuuint64_t)BKB * 2, (cuuint64_t)op->R * BKB * 2};
    cuuint32_t box[3] = {BKB, BM, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode_fn()(&op->tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, op->buf, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        dfree(mem, op->buf);
        op->buf = nullptr;
        *err = "Davidson operand tensor map: error " + std::to_string((int)r);
        return HB_ERR_CUDA;
    }
    return HB_OK;
}

void dense_operand_free(hb_ctx *mem, DenseOperand *op) {
    if (op->buf) dfree(mem, op->buf);
    op->buf = nullptr;
}

void dense_operand_fill(const DenseOperand &op, int S, const double *X1, int64_t ld1, int K1, const double *X2,
                        int64_t ld2, int K2, int64_t rows, cudaStream_t s) {
    if (rows <= 0) return;
    slice_rows2_kernel<<<(unsigned)rows, 1024, 0, s>>>(X1, ld1, K1, X2, ld2, K2, op.Kpad, S, op.R,
                                                       (__nv_bfloat16 *)op.buf);
}

int dense_splits(int64_t M, int64_t N, int kb_total, int *kb_per_split) {
    const int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    const int kpc = KCHUNK / BKB;
    const int max_split = (kb_total + kpc - 1) / kpc;
    int ns = (int)std::max<int64_t>(1, std::min<int64_t>(max_split, (3 * 152 + tiles - 1) / tiles));
    int per = (kb_total + ns - 1) / ns;
    per = (per + kpc - 1) / kpc * kpc;
    *kb_per_split = per;
    return (kb_total + per - 1) / per;
}

int dense_split_gemm(int S, const DenseOperand &A, int64_t M, const DenseOperand &B, int64_t N, int kb_total,
                     float2 *part, double *Y, int64_t ldy, int *err, cudaStream_t s) {
    if (M <= 0 || N <= 0 || kb_total <= 0) return 0;
    static bool attr[MAXS + 1] = {false};
    const int bytes = S * SLOT + 2048;
    DenseArgs a;
    a.M = (int)M; a.N = (int)N;
    a.kb_total = kb_total;
    const int nsplit = dense_splits(M, N, kb_total, &a.kb_per_split);
    a.a_planes = A.planes; a.b_planes = B.planes;
    a.part = part;
    a.err = err;
    const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)nsplit);
#define HB_DENSE(SS)                                                                                    \
    do {                                                                                                \
        if (!attr[SS]) {                                                                                \
            cudaFuncSetAttribute(dense_split_kernel<SS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); \
            attr[SS] = true;                                                                            \
        }                                                                                               \
        dense_split_kernel<SS><<<grid, NTHREADS, bytes, s>>>(A.tm, B.tm, a);                            \
    } while (0)
    switch (S) {
        case 2: HB_DENSE(2); break;
        case 3: HB_DENSE(3); break;
        case 4: HB_DENSE(4); break;
        case 5: HB_DENSE(5); break;
        default: HB_DENSE(6); break;
    }
#undef HB_DENSE
    const int64_t tot = M * N;
    dense_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, nsplit, (int)M, (int)N, Y, ldy);
    return 2;
}

void release_mixed(hb_ctx *ctx) {
    if (!ctx->mixed) return;
    if (!ctx->mixed->borrowed_panel) {
        dfree(ctx, ctx->mixed->panel_slices);
        dfree(ctx, ctx->mixed->pdiag);
    }
    delete ctx->mixed;
    ctx->mixed = nullptr;
}
