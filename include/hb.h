/*
 * hb.h -- C ABI of the GB300 close-coupling Hamiltonian build.
 *
 * The library builds the contracted (N+1)-electron scattering Hamiltonian of
 * the close-coupling expansion (Eq. 1 of Al-Refaie & Tennyson, "A parallel
 * algorithm for Hamiltonian matrix construction in electron-molecule
 * collision calculations: MPI-SCATCI") with Tennyson's structured algorithm
 * (Section 2.1: bitstring Slater-Condon rules, prototype symbols, contraction
 * with the target CI coefficients, Eq. 6-8, and expansion over continuum
 * orbitals), and finds its lowest eigenpairs (Section 3.2.2, Davidson).
 *
 * Conventions
 * -----------
 * Orbitals: spatial orbitals 0..n_to-1 are target orbitals, n_to..n_to+n_co-1
 *   continuum orbitals.  Continuum index j (0..n_co-1) is orbital n_to+j.
 * Determinants: 2*n_words uint64 words, words [0, W) the alpha string and
 *   [W, 2W) the beta string; bit p of a string is target orbital p.  The
 *   (N+1)-electron determinant of a target determinant D and continuum orbital
 *   j is the canonically ordered product of creation operators over all alpha
 *   spin orbitals (target, then continuum) followed by all beta ones, so the
 *   continuum spin orbital sits above every target orbital of its spin and
 *   every phase and integral label is independent of j (prototyping).
 * Integrals (chemists' notation, real, 8-fold symmetric; pair(p,q) =
 *   p(p+1)/2+q for p >= q, Pt = n_to(n_to+1)/2):
 *     h[(n_to+n_co)^2]                 one-electron, row-major, symmetric
 *     eri_tttt[Pt][Pt]                 (pq|rs), four target indices
 *     eri_tttc[Pt][n_to*n_co]          (pq|r j) at [pair(p,q)][r*n_co + j]
 *     eri_ttcc[Pt][n_co*n_co]          (pq|j k) at [pair(p,q)][j*n_co + k]
 *     eri_tctc[n_to*n_co][n_to*n_co]   (r j|s k) at [r*n_co + j][s*n_co + k]
 *   No other class is needed: an (N+1)-electron function holds at most one
 *   continuum electron, so at most two continuum indices occur (Section 2.1).
 * Basis order of the result: for each target group g (a target symmetry),
 *   for each state n, for each continuum orbital j of its range (n-major);
 *   then the L2 functions.  Group g starts at row group_offset(g).
 *
 * Results (hb_blocks, all caller-owned device memory):
 *   Hcc  [Dc][Dc]      continuum-continuum classes 1,3,5,6,7, full symmetric
 *   Hlc  [n_l2][Dc]    class 4, L2 row l against contracted column (g,n,j);
 *                      this is the lower-triangle block of the matrix
 *   CSR  row_ptr[n_l2+1] (int64), col[nnz] (int32), val[nnz] (double):
 *                      classes 2 and 8, the full symmetric L2 x L2 block with
 *                      one entry per pair within a double excitation (each
 *                      entry below the diagonal is a copy of its mirror)
 *   Dc = contracted dimension, dim = Dc + n_l2.
 *
 * Errors: every call returns an int status (HB_OK = 0); no exception crosses
 * the ABI and nothing aborts.  hb_last_error(ctx) (or hb_last_error(NULL)
 * for calls without a context) returns a message for the last failure.
 * Streams: `stream` is a cudaStream_t passed as void*; NULL means the legacy
 * default stream.  Work is enqueued on it; calls that must read a device
 * result (counts, convergence) synchronise that stream before returning.
 */
#ifndef HB_H
#define HB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HB_OK = 0,
    HB_ERR_INVALID_ARG = 1,
    HB_ERR_CUDA = 2,
    HB_ERR_OOM = 3,
    HB_ERR_TIMEOUT = 4,
    HB_ERR_NOT_CONVERGED = 5,
    HB_ERR_UNSUPPORTED = 6
};

enum { HB_FP64 = 0, HB_MIXED = 1 };
enum { HB_PRECOND_DIAG = 0, HB_PRECOND_MLP = 1 };
/* OR'ed into hb_diag's precond: the block products H V on the tensor cores
   in split-bf16 form (7 bits a slice, 6 slices a value, exact FP32 chunks);
   the Rayleigh-Ritz projection and the orthogonalisation stay FP64. */
enum { HB_DIAG_TENSOR = 0x100 };
enum { HB_SPIN_ALPHA = 0, HB_SPIN_BETA = 1 };

typedef struct hb_ctx hb_ctx;

/* One target symmetry (Eq. 2): phi_n = sum_m c[m][n] D_m, coupled to the
   contiguous continuum range [cont_first, cont_first + cont_count).
   energy (host [n_state], or NULL): target-state energies for the
   target-energy substitution of Section 3.1.  When given (for every group or
   for none), the CI vectors are taken to be eigenvectors of the N-electron
   target Hamiltonian H^N (+ e_core on its diagonal), and the target-only part
   of the continuum-continuum block, <phi_gn|H^N + e_core|phi_g'n'>, is
   delta_gg' delta_nn' energy[n] instead of the Eq. 8 sum over the target-only
   integrals.  hb_target_diag returns such energies and CI vectors. */
/* Spin-adapted groups (Eq. 2 with configuration state functions as the
   eta_im): with n_csf > 0, CSF i is sum_k csf_coef[k] D[csf_det[k]] over
   csf_ptr[i] <= k < csf_ptr[i+1] (determinants of this group's list) and ci
   is [n_csf][n_state] over the CSFs.  hb_init expands the CI vectors over the
   determinants on the device (one more contraction level ahead of Eq. 8).
   Groups may share determinants only when they have the same determinant set
   and the same continuum range and are adjacent in the list (for instance a
   singlet and a triplet target over the same configurations, coupled to the
   same continuum: classes 5 and 6 between target spins); the library builds
   them as one group whose states are the groups' states in order, which is
   the same row layout. */
typedef struct {
    int32_t n_det;
    int32_t n_state;
    const uint64_t *dets;   /* host, [n_det][2*n_words] */
    const double *ci;       /* host, [n_det][n_state] (or [n_csf][n_state]), row-major */
    int32_t cont_first;
    int32_t cont_count;
    const double *energy;   /* host, [n_state], or NULL */
    int32_t n_csf;          /* 0: ci is over the determinants */
    const int32_t *csf_ptr; /* host, [n_csf + 1] (n_csf > 0) */
    const int32_t *csf_det; /* host, [csf_ptr[n_csf]], indices into dets */
    const double *csf_coef; /* host, [csf_ptr[n_csf]] */
} hb_group;

/* The problem of Eq. 1: orbitals, integrals, target groups, L2 functions.
   All pointers are host pointers; hb_init copies what it needs. */
typedef struct {
    int32_t n_to, n_co;     /* target and continuum spatial orbitals */
    int32_t n_elec;         /* N, target electrons (the system has N+1) */
    int32_t n_words;        /* W, uint64 words per spin string (1..4) */
    int32_t cont_spin;      /* spin of the continuum electron, HB_SPIN_* */
    const double *h;
    const double *eri_tttt, *eri_tttc, *eri_ttcc, *eri_tctc;
    int32_t n_groups;
    const hb_group *groups;
    int32_t n_l2;
    const uint64_t *l2_dets;  /* host, [n_l2][2*n_words], N+1 electrons */
    double e_core;            /* constant added to the Hamiltonian (0 if none) */
    const int32_t *orb_irrep; /* host, [n_to + n_co], or NULL: the spatial symmetry of every orbital
                                 (irreducible representation 0..7 of an abelian point group whose
                                 product is XOR, as for D2h and its subgroups).  With it the
                                 integrals must vanish unless the XOR of their four orbitals' irreps
                                 is 0 (checked on the device when validating), and every group's
                                 continuum range must lie within one irrep.  The expansion panel
                                 then keeps, for each continuum pair, only the labels of its
                                 symmetry (about an eighth of them): less memory and work, the
                                 same results up to the order of the sums. */
} hb_problem;

typedef struct {
    int32_t split_slices;     /* mixed path: bf16 slices per operand (2..6), 0 = default (6) */
    int32_t validate;         /* 0 = skip the O(n^2) input checks */
    int32_t autotune;         /* 1 = time the launch-shape candidates on the first build
                                 (results are bit-identical for every candidate) */
    int32_t split_tile;       /* 0 = chosen; 3, 4, 5: tensor-core tiles of (128 >> v) j x (1 << v) j' */
    int32_t class4_states;    /* 0 = chosen; 4, 8, ..., 32, 40, 48, 56, 64: target states per pass of the
                                 double-float class-4 kernel */
    int32_t class4_threads;   /* 0 = chosen; 32, 64, 128: continuum orbitals per class-4 block */
    int32_t class4_path;      /* mixed build, class 4: 0 = tensor cores for groups of 32..64 states and
                                 the double-float kernel for the rest; 1 = the double-float kernel
                                 only; 2 = tensor cores for every group of 1..64 states */
    int32_t mlp_stall_iters;  /* HB_PRECOND_MLP: the learned factor is dropped for the rest of a solve
                                 when the largest wanted residual has not fallen by 2^mlp_stall_log2
                                 over the last mlp_stall_iters iterations; 0 = 10 (1..1000) */
    int32_t mlp_stall_log2;   /* 0 = 1, i.e. halved (1..60) */
    int32_t diag_basis;       /* hb_diag: the basis holds at most diag_basis blocks of b vectors
                                 (b = k + min(16, max(4, k / 2))) before a thick restart to 2b;
                                 0 = 6 (3..10) */
    int32_t split_cols;       /* 0 = chosen: below 2048 labels per merged block from its columns
                                 (state pairs n, n'): 32 up to 32, 64 up to 64, else 128; from 2048
                                 labels on, 128.  32, 64, 128 force that width of the tensor-core
                                 tiles.  Results are bit-identical for every width that keeps the
                                 K stage (below) */
    int32_t split_kstage;     /* 0 = chosen: K stages of 64 for 128-column tiles from 2048 labels on,
                                 of 32 otherwise; 32 or 64 forces it for 128-column tiles (narrower
                                 tiles always use 32).  The two orders of the products round the
                                 FP32 accumulator of the slice pairs i + l >= 3 (terms below 2^-21
                                 of the largest products) differently, so results agree within the
                                 mixed path's error bound, not bit for bit; every other shape
                                 option keeps the bits */
    int32_t reserved[4];
} hb_options;

typedef struct {
    int64_t dim, contracted_dim, n_l2, l2_nnz;
    int64_t tt_pairs;         /* target x target pairs within a double excitation */
    int64_t tl2_pairs;        /* target x L2 pairs within a double excitation */
    int64_t n_labels;         /* K: labels of the expansion contraction */
    int64_t device_bytes;     /* device memory held by the context */
    int32_t n_groups;
    int32_t n_words;
    int64_t workspace_bytes;  /* the last hb_workspace_size result (0 before the first call) */
} hb_layout;

typedef struct {
    double *Hcc;
    double *Hlc;
    int64_t *l2_row_ptr;
    int32_t *l2_col;
    double *l2_val;
} hb_blocks;

typedef struct {
    float ms_total;           /* build: enqueue to completion on the stream */
    /* The stages run on two streams (target side then expansion; class 4 and
       the L2 rows beside them), so these spans overlap and their sum exceeds
       ms_total.  With class 4 on the tensor cores the expansion waits for it,
       and ms_expand includes that wait. */
    float ms_target;          /* classification + target-side contraction */
    float ms_expand;          /* continuum-continuum expansion */
    float ms_class4;          /* class-4 classification and kernels */
    float ms_l2;              /* classes 2 and 8 */
    float ms_expand_gemm;     /* dominant kernel alone (expansion contraction) */
    int32_t expand_launches;
    int32_t kernel_launches;  /* kernels launched by the call */
    double expand_flops;      /* algorithmic flops of the expansion */
    int32_t iterations;       /* hb_diag */
    int32_t mlp_fallbacks;
    double max_residual;
    float ms_matvec;
    float ms_rr;              /* hb_diag: host time of the small eigenproblems */
    double expand_tensor_flops;  /* mixed: bf16 tensor flops of the split products */
    float ms_gram;            /* hb_diag: projections (device sums and their copy to the host) */
    float ms_combine;         /* hb_diag: basis combinations (coefficients to the device, kernel) */
    float ms_class4_kernel;   /* the class-4 kernels after their classification (part of ms_class4) */
    int32_t fp64_iterations;  /* hb_diag: iterations with FP64 products after the convergence check */
    float mlp_loss;           /* hb_mlp_train: loss of the last window */
    int32_t proj_gflop;       /* hb_diag: FP64 GFLOP of the projections and basis combinations
                                 (the Gram sums, norms, project-outs and combines: 2 flops per term) */
} hb_stats;

/* Excitation record of one determinant pair (row, col), see hb_classify. */
typedef struct {
    int32_t row, col;
    int16_t hole[2];          /* bit positions (spin*64*W + orbital) in col only */
    int16_t part[2];          /* bit positions in row only; -1 if unused */
    int8_t degree;
    int8_t phase;             /* +1 / -1 */
    int16_t pad[3];
} hb_pair;

/* Validate and copy a problem (Eq. 1-2), stage it on the current device and
   build the continuum-continuum integral panels.  Also finds the sparsity
   pattern of every class and, for the L2 x L2 block, the position of each
   entry's mirror.  Allocates the device memory the context needs (reported
   by hb_query).  Errors: HB_ERR_INVALID_ARG for
   inconsistent input (electron counts, spins, duplicate determinants, ranges,
   non-finite integrals, orbital counts beyond 16-bit labels), HB_ERR_OOM,
   HB_ERR_CUDA, HB_ERR_UNSUPPORTED (n_words > 4). */
int hb_init(hb_ctx **ctx, const hb_problem *p, const hb_options *o, void *stream);

/* Sizes of the result and of the context (Section 2.2 classes). */
int hb_query(const hb_ctx *ctx, hb_layout *out);

/* Caller-owned workspace (no counterpart in the paper).  hb_init allocates
   the staged problem (integrals, determinants, CI vectors, the expansion
   panel and the per-group-pair buffers whose sizes come from its
   classification pass; hb_layout.device_bytes).  Everything a build or a
   solve sets up after that (the build plan, the double-float copies, the
   tensor-core slices and class-4 tables, the Davidson vectors and scratch,
   the learned factors) is allocated on first use with cudaMalloc, or, once a
   workspace is set, carved out of it: builds and solves then allocate no
   device memory.

   hb_workspace_size measures the bytes: the build set-up for `precision`
   (HB_FP64, HB_MIXED, or -1 for none) is made once under a byte count and
   released, and the solver's bytes for diag_k eigenpairs (0: none) with the
   given precond flags (HB_DIAG_TENSOR, HB_PRECOND_MLP) are added; the result
   includes 16 MiB and 1.6 % for the autotuner's timing buffers and alignment.
   It is also reported as hb_layout.workspace_bytes.  It must be called before
   hb_set_workspace; it synchronises `stream`.

   hb_set_workspace gives the context a device buffer of `bytes` bytes that the
   caller owns and keeps alive until hb_destroy (or until the context is no
   longer used).  Whatever a previous build or solve had set up is released
   first.  A build or solve whose set-up does not fit returns HB_ERR_OOM.  A
   workspace can be set once per context.  Errors: HB_ERR_INVALID_ARG (NULL,
   a workspace already set), HB_ERR_CUDA. */
int hb_workspace_size(hb_ctx *ctx, int32_t precision, int32_t diag_k, int32_t precond, int64_t *bytes,
                      void *stream);
int hb_set_workspace(hb_ctx *ctx, void *dev_ptr, size_t bytes);

/* First row of target group g in the contracted basis. */
int64_t hb_group_offset(const hb_ctx *ctx, int32_t g);

/* Build every class (1-8) into the caller's device buffers.  precision:
   HB_FP64 (double arithmetic throughout) or HB_MIXED: the continuum-continuum
   contraction (Eq. 7), and class 4 (Eq. 5) of groups of 32..64 states (see
   hb_options.class4_path), on bf16 tensor cores with split operands, exact
   FP32 accumulation and double-float recovery; the target-side contraction
   and the other class-4 groups in double-float on the FP32 pipes; classes 2
   and 8 in FP64.  The results are written as FP64.  `st` may be NULL.
   Errors: HB_ERR_INVALID_ARG, HB_ERR_OOM, HB_ERR_CUDA, HB_ERR_TIMEOUT (a
   bounded wait of a tensor-core kernel gave up). */
int hb_build_blocks(hb_ctx *ctx, int32_t precision, const hb_blocks *out, hb_stats *st,
                    void *stream);

/* Lowest k eigenpairs of the built matrix by block Davidson (Section 3.2.2)
   to ||H x - lambda x||_2 <= tol for each pair.  evals: host [k]; evecs:
   device [dim][k] row-major or NULL; v0: device [dim][k] start vectors or
   NULL (unit vectors at the smallest diagonal entries).  precond:
   HB_PRECOND_DIAG, or HB_PRECOND_MLP after hb_mlp_set, optionally OR
   HB_DIAG_TENSOR (block products on the tensor cores).  With HB_PRECOND_MLP
   the solve falls back to the diagonal preconditioner for good when the
   largest wanted residual has not halved over 10 iterations (counted in
   st->mlp_fallbacks).  Returns
   HB_ERR_NOT_CONVERGED after max_iter iterations (evals then hold the current
   Ritz values). */
int hb_diag(hb_ctx *ctx, const hb_blocks *H, int32_t k, double tol, int32_t max_iter,
            int32_t precond, const double *v0, double *evals, double *evecs, hb_stats *st,
            void *stream);

/* Target states of group g of a problem (Section 3.1 with the classes 2/8
   machinery of Section 2.2): the lowest k eigenpairs of the N-electron target
   Hamiltonian H^N + e_core over the group's determinants.  H^N is built on the
   device by the L2-L2 Slater-Condon kernels applied to the N-electron
   determinants (CSR, FP64) and solved by hb_diag's block Davidson with the
   diagonal preconditioner to ||H^N c - E c||_2 <= tol for each pair.  Only
   the problem's orbital counts, h, eri_tttt, e_core and the group's
   determinants are read.  energies: host [k], ascending; ci: host [n_det][k],
   row-major, orthonormal columns (each column's sign fixed so that its
   largest-magnitude entry is positive): ready to be passed as the group's ci
   and energy for the target-energy substitution.  st (or NULL) receives the
   solve's statistics.  The call allocates and frees its own device memory.
   Errors: HB_ERR_INVALID_ARG (g out of range, k < 1 or k > n_det, NULL
   outputs), HB_ERR_NOT_CONVERGED after max_iter iterations (outputs then hold
   the current Ritz pairs), HB_ERR_OOM, HB_ERR_CUDA. */
int hb_target_diag(const hb_problem *p, int32_t g, int32_t k, double tol, int32_t max_iter, double *energies,
                   double *ci, hb_stats *st, void *stream);

/* Sharded build over nranks processes (Section 3.1, the distributed
   prototype contraction with the reduction of Eq. 11, and Section 3.2, the
   distributed matrix).  Rank r of R:
     1. hb_build_contract: the target-side contraction (Eq. 8) over the bra
        determinants [ndet r / R, ndet (r + 1) / R) of every group pair gives
        this rank's share of the contracted coefficient rows, written to
        `partial` (device, hb_shard_coef_len doubles: for every group pair in
        order, its state pairs x the padded label count);
     2. the caller sums the partials of all ranks (an all-reduce, NCCL for
        instance) into `reduced`, the same on every rank;
     3. hb_build_expand: with the reduced rows, this rank's share of the rest:
        the continuum-continuum tiles r, r + R, ... of Eq. 7 (rank 0 also the
        rows with j == j' on the mixed path), the class-4 rows and the L2 rows
        [n_l2 r / R, n_l2 (r + 1) / R) (an L2 entry below the diagonal is
        written by the rank that owns its mirror's row).
   Every element of the result is written by exactly one rank; what a rank
   does not write it leaves as it was, so the ranks' zero-initialised outputs
   add up to the whole matrix (the L2 row pointers included).  The contraction
   sums of a rank run in the order of the one-rank build; the reduction adds
   the ranks' partial sums, so results agree with hb_build_blocks to the
   rounding of that reordering.  With the target-energy substitution rank 0
   adds the energies.  The plan of the share is kept for the next call.
   Errors: HB_ERR_INVALID_ARG (rank outside 0..nranks-1, NULL buffers),
   HB_ERR_OOM, HB_ERR_CUDA, HB_ERR_TIMEOUT. */
int hb_shard_coef_len(const hb_ctx *ctx, int64_t *len);
int hb_build_contract(hb_ctx *ctx, int32_t precision, int32_t rank, int32_t nranks, double *partial, hb_stats *st,
                      void *stream);
int hb_build_expand(hb_ctx *ctx, int32_t precision, int32_t rank, int32_t nranks, const double *reduced,
                    const hb_blocks *out, hb_stats *st, void *stream);

/* Stage a problem whose orbitals and integrals are those of `base` (for
   instance another spatial-symmetry or spin-coupling block of the same
   molecule): the integrals, the expansion panel and its tensor-core slices are
   borrowed from `base`, which must outlive this context.  The caller
   guarantees that p's integral arrays equal base's (only their shapes are
   checked). */
int hb_init_shared(hb_ctx **ctx, const hb_problem *p, const hb_options *o, hb_ctx *base, void *stream);

/* Batched build of n staged contexts into outs[0..n) (Section 2.2 classes for
   every block).  The contexts must share the target orbital space (n_words,
   n_to).  Every stage of the build is one grouped launch over the group pairs
   of all contexts; the group pairs of any context that read the same
   continuum rectangle of the same panel share one expansion GEMM (Eq. 7).
   Creation times the launch-shape candidates once on the batch's own tasks
   (results are bit-identical for every candidate), then captures the whole
   set as a CUDA graph that hb_batch_launch replays with a single launch.  The
   blocks in outs are baked into the graph and must stay allocated.  st of
   hb_batch_launch (or NULL) receives the per-stage times of the replay. */
typedef struct hb_batch hb_batch;
int hb_batch_create(hb_batch **b, hb_ctx *const *ctxs, int32_t n, int32_t precision, const hb_blocks *outs,
                    void *stream);
int hb_batch_launch(hb_batch *b, hb_stats *st, void *stream);
int hb_batch_nodes(const hb_batch *b);
void hb_batch_destroy(hb_batch *b);

/* The launch shapes a batch (or a context's own build plan) uses, as text
   into buf (NUL-terminated, truncated to len).  Returns the full length, -1
   on a NULL argument.  No counterpart in the paper: reports the autotuner. */
int32_t hb_batch_report(const hb_batch *b, char *buf, int32_t len);
int32_t hb_tuning_report(const hb_ctx *ctx, char *buf, int32_t len);

/* Excitation classification (Section 2.1) of every pair (a, b) of two
   determinant lists on the device.  mode 0: equal electron counts, degree =
   popcount(a ^ b) / 2; mode 1: b holds N-electron target determinants and a
   holds (N+1)-electron ones, the pair being (b + continuum electron of spin
   cont_spin, a), degree = popcount(b & ~a) + 1.  Pairs with degree <= max_degree
   (and b <= a when lower != 0) are written to pairs[] ordered by (a, b), with
   row = a, col = b.  row_ptr (device, n_a + 1) receives the CSR offsets.  The
   total goes to *total; if it exceeds cap nothing is written to pairs and
   HB_ERR_INVALID_ARG is returned.  Phase = <row| a+_p1 a+_p2 a_h2 a_h1 |col>
   (or a+_p a_h) with holes in col only and particles in row only, ascending
   in the canonical order; for mode 1 the continuum electron is a particle
   and is not listed. */
int hb_classify(const uint64_t *a, int32_t n_a, const uint64_t *b, int32_t n_b,
                int32_t n_words, int32_t mode, int32_t cont_spin, int32_t max_degree,
                int32_t lower, int64_t *row_ptr, hb_pair *pairs, int64_t cap,
                int64_t *total, void *stream);

/* Allocation-free variant of hb_classify.  The paper has no counterpart: it
   exists for callers that cannot allocate device memory (a host framework
   that owns the allocator, a plug-in that may not call cudaMalloc after
   start-up, a real-time loop that cannot afford an allocation's implicit
   synchronisation) and so cannot provide hb_classify's row_ptr buffer.  The
   row offsets live instead in a static device array of HB_NOALLOC_MAX_ROWS + 1
   int64 values (2 MiB) that every GPU loading the library holds until the
   process exits.  Same arguments and results as hb_classify without row_ptr;
   n_a > HB_NOALLOC_MAX_ROWS returns HB_ERR_INVALID_ARG.  The function calls no
   allocating routine.  Its first call on a device looks up the array's device
   address (cudaGetSymbolAddress) with that device current; make that first
   call before any stream capture.  The address is kept for the life of the
   process: a cudaDeviceReset of that device invalidates it, and the entry
   point must not be called on that device after such a reset.  All calls
   share the array, so calls whose work overlaps on the GPU race: serialise
   them.  Errors are reported through hb_last_error(NULL). */
#define HB_NOALLOC_MAX_ROWS 262144
int hb_classify_noalloc(const uint64_t *a, int32_t n_a, const uint64_t *b, int32_t n_b,
                        int32_t n_words, int32_t mode, int32_t cont_spin, int32_t max_degree,
                        int32_t lower, hb_pair *pairs, int64_t cap, int64_t *total, void *stream);

/* ---- learned Davidson preconditioner (a small MLP, not in the paper) ---- */

typedef struct {
    int32_t n_in, width;      /* input features, hidden width */
    const float *w1, *b1;     /* host [width][n_in], [width] */
    const float *w2, *b2;     /* host [width][width], [width] */
    const float *w3, *b3;     /* host [1][width], [1] */
} hb_mlp_weights;

/* Weights of the network used by hb_diag with HB_PRECOND_MLP: 8 inputs,
   width 64 (w1 [64][8], b1 [64], w2 [64][64], b2 [64], w3 [64], b3 [1]);
   stored as FP16, biases FP32.  The factor for row i and Ritz value theta is
   w = 256^tanh(o), o = w3 . relu(w2 relu(w1 f + b1) + b2) + b3, applied as
   t_i = w r_i / (H_ii - theta).  A non-finite factor falls back to 1. */
int hb_mlp_set(hb_ctx *ctx, const hb_mlp_weights *w);

/* Number of packed parameters (w1, b1, w2, b2, w3, b3 in that order) for
   n_in = 8, width = 64 (4801); -1 for any other shape. */
int hb_mlp_param_count(int32_t n_in, int32_t width);

/* Device scratch needed by hb_mlp_loss_grad for n samples. */
int64_t hb_mlp_workspace_bytes(int64_t n);

/* Training step pieces, all device pointers.  For samples i with features
   feats[i][8] and targets a_i, b_i: loss = mean_i (w(f_i) a_i - b_i)^2 and its
   gradient with respect to the packed parameters (weights rounded to FP16 in
   the forward pass, FP32 accumulation, fixed-order sums). */
int hb_mlp_loss_grad(const float *params, const float *feats, const float *a, const float *b, int64_t n,
                     float *grads, float *loss, void *work, void *stream);

/* One Adam update (beta1 0.9, beta2 0.999, eps 1e-8) of n_param parameters. */
int hb_mlp_adam(int64_t n_param, float *params, const float *grads, float *m, float *v, int32_t step,
                float lr, void *stream);

/* A training set of the learned preconditioner (device arrays): features
   feats [n][8], targets a [n], b [n] (loss of hb_mlp_loss_grad), and the
   schedule: `steps` Adam updates (learning rate lr), each over the next window
   of `batch` samples, wrapping around. */
typedef struct {
    int64_t n;
    const float *feats;
    const float *a, *b;
    int64_t batch;
    int32_t steps;
    float lr;
} hb_mlp_dataset;

/* Adam training of the packed parameters `params` (device, in place) on the
   data set d; the trained network then becomes the context's preconditioner
   network (as hb_mlp_set).  Scratch comes from the context's memory (its
   workspace when one is set).  st (or NULL): iterations = steps, mlp_loss =
   the last window's loss.  Errors: HB_ERR_INVALID_ARG, HB_ERR_OOM, HB_ERR_CUDA.
   Not in the paper: the learned preconditioner. */
int hb_mlp_train(hb_ctx *ctx, const hb_mlp_dataset *d, float *params, hb_stats *st, void *stream);

/* The same loop without a context: params (device, in place), the data set as
   arrays, the last window's loss into *last_loss (host, may be NULL); the
   scratch is allocated and freed by the call. */
int hb_mlp_train_params(float *params, const float *feats, const float *a, const float *b, int64_t n,
                        int64_t batch, int32_t steps, float lr, float *last_loss, void *stream);

/* Factors w(f_i) for n feature rows (device). */
int hb_mlp_predict(const float *params, const float *feats, int64_t n, float *out, void *stream);

/* Features of every row of the built matrix for q Ritz values theta (host):
   feats (device) [q][dim][8], as hb_diag computes them. */
int hb_diag_features(hb_ctx *ctx, const hb_blocks *H, const double *theta, int32_t q, float *feats,
                     void *stream);

/* A text description of a context (sizes of every class of Section 2.2,
   the target groups, device memory, the build plan's launch shapes) written
   to the file at `path`.  Errors: HB_ERR_INVALID_ARG (NULL argument or the
   file cannot be written). */
int hb_dump(const hb_ctx *ctx, const char *path);

const char *hb_last_error(const hb_ctx *ctx);
void hb_destroy(hb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* HB_H */
