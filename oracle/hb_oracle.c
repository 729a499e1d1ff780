/*
 * hb_oracle.c -- plain FP64 CPU oracle of the structured close-coupling
 * Hamiltonian build (Tennyson's prototype / contract / expand algorithm).
 *
 * ORACLE / TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header
 * or table with the CUDA library; both read the same seeded inputs.
 *
 * What it computes, in the paper's order:
 *   - Section 2.1, bitstring Slater-Condon rules (Scemama-Giner): excitation
 *     degree from XOR + popcount, holes/particles from the bits, phase from
 *     the number of occupied spin orbitals between hole and particle (masks
 *     built without the shift-by-64 trap that the paper reports fixing).
 *   - Eq. 6: each determinant pair gives a symbolic list sum_a C^a X(I^a)
 *     with integral labels of four 16-bit orbital indices packed in 64 bits.
 *   - Prototyping: the continuum electron is a placeholder orbital above all
 *     target orbitals of its spin; two prototypes are evaluated, "same
 *     continuum orbital" (j = j') and "different continuum orbitals"; labels
 *     hold placeholders and do not depend on j.
 *   - Eq. 8: the prototype coefficients are contracted with the target CI
 *     vectors, D^b = sum_{m m'} c_mn c_m'n' C^a, labels unchanged.
 *   - Eq. 7: the labels are expanded over the continuum orbitals j, j' and
 *     the integral function X looks each one up.
 *   - Eq. 5 / class 4: the same for one continuum placeholder against an L2
 *     determinant, contracted over m only.
 *   - classes 2 and 8: L2-L2 elements evaluated directly.
 *
 * Conventions (inputs):
 *   spatial orbitals 0..n_to-1 target, n_to..n_to+n_co-1 continuum;
 *   determinant = 2W uint64 words, alpha string then beta string;
 *   spin-orbital canonical order: all alpha (target, then continuum), then
 *   all beta;  bit position of target (p, spin) = spin*64*W + p;
 *   integral class arrays as documented in the Python generator.
 * All arithmetic is double precision; no blocking, fusion or reordering
 * beyond the order stated above.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXW 8          /* words per spin in extended strings */
#define ORC_CHUNKS 64       /* fixed bra-determinant chunks of the contraction */
#define ORC_ONE_E 0xFFFFu   /* marker in slots r,s of a one-electron label */
#define ORC_OVERLAP 0xFFFEu /* marker label for the overlap (core energy) term */

typedef struct {
    int32_t n_to, n_co, n_elec, W, cont_spin;
    const double *h, *tttt, *tttc, *ttcc, *tctc;
    int32_t n_groups;
    const int32_t *g_ndet, *g_nstate, *g_cfirst, *g_ccount;
    const uint64_t *const *g_dets;
    const double *const *g_ci;
    int32_t n_l2;
    const uint64_t *l2;
    double e_core;
    /* target-energy substitution (Section 3.1): per group, the state
       energies, or NULL when the target-only part is the Eq. 8 sum */
    const double *const *g_energy;
} orc_problem;

static int popc64(uint64_t x) { return __builtin_popcountll(x); }

static int64_t pairidx(int p, int q) {
    if (p < q) { int t = p; p = q; q = t; }
    return (int64_t)p * (p + 1) / 2 + q;
}

/* ------------------------------------------------------------------------ */
/* integral function X                                                       */
/* ------------------------------------------------------------------------ */

static double orc_one(const orc_problem *P, int p, int q) {
    int n = P->n_to + P->n_co;
    return P->h[(int64_t)p * n + q];
}

/* (pq|rs), global spatial indices, at most two continuum indices */
static double orc_two(const orc_problem *P, int p, int q, int r, int s) {
    const int nt = P->n_to, nc = P->n_co;
    const int64_t Pt = (int64_t)nt * (nt + 1) / 2, NTC = (int64_t)nt * nc;
    int cp = p >= nt, cq = q >= nt, cr = r >= nt, cs = s >= nt;
    int ncont = cp + cq + cr + cs;
    if (ncont == 0) return P->tttt[pairidx(p, q) * Pt + pairidx(r, s)];
    if (ncont == 1) {
        if (cp || cq) { int t; t = p; p = r; r = t; t = q; q = s; s = t; t = cp; cp = cr; cr = t; t = cq; cq = cs; cs = t; }
        if (cr) { int t = r; r = s; s = t; }
        return P->tttc[pairidx(p, q) * NTC + (int64_t)r * nc + (s - nt)];
    }
    if (ncont == 2) {
        if (cp && cq) return P->ttcc[pairidx(r, s) * ((int64_t)nc * nc) + (int64_t)(p - nt) * nc + (q - nt)];
        if (cr && cs) return P->ttcc[pairidx(p, q) * ((int64_t)nc * nc) + (int64_t)(r - nt) * nc + (s - nt)];
        int t1 = cp ? q : p, c1 = cp ? p : q;
        int t2 = cr ? s : r, c2 = cr ? r : s;
        return P->tctc[((int64_t)t1 * nc + (c1 - nt)) * NTC + (int64_t)t2 * nc + (c2 - nt)];
    }
    return NAN; /* never needed with a single continuum electron */
}

/* ------------------------------------------------------------------------ */
/* bitstrings: Section 2.1                                                   */
/* ------------------------------------------------------------------------ */

/* mask of bits [lo, hi) inside one 64-bit word, 0 <= lo <= hi <= 64 */
static uint64_t range_mask(int lo, int hi) {
    uint64_t up = (hi >= 64) ? ~0ull : ((1ull << hi) - 1ull);
    uint64_t dn = (lo <= 0) ? 0ull : ((lo >= 64) ? ~0ull : ((1ull << lo) - 1ull));
    return up & ~dn;
}

/* number of set bits strictly between positions a and b of a string of nw words */
static int popc_between(const uint64_t *D, int nw, int a, int b) {
    if (a > b) { int t = a; a = b; b = t; }
    int cnt = 0;
    for (int w = 0; w < nw; ++w) {
        int lo = a + 1 - 64 * w, hi = b - 64 * w;
        if (hi <= 0 || lo >= 64) continue;
        if (lo < 0) lo = 0;
        if (hi > 64) hi = 64;
        if (lo < hi) cnt += popc64(D[w] & range_mask(lo, hi));
    }
    return cnt;
}

typedef struct {
    int degree;
    int holes[2];  /* bit positions occupied in ket J only, ascending */
    int parts[2];  /* bit positions occupied in bra I only, ascending */
    int phase;     /* <I| a+_p1 a+_p2 a_h2 a_h1 |J> (or a+_p a_h) */
} orc_exc;

/* Excitation between two strings of nw words (all spins concatenated). */
static void orc_excitation(int nw, const uint64_t *I, const uint64_t *J, orc_exc *e) {
    int nd = 0;
    for (int w = 0; w < nw; ++w) nd += popc64(I[w] ^ J[w]);
    e->degree = nd / 2;
    e->phase = 1;
    e->holes[0] = e->holes[1] = e->parts[0] = e->parts[1] = -1;
    if (e->degree > 2 || e->degree == 0) return;
    int nh = 0, np = 0;
    for (int w = 0; w < nw; ++w) {
        uint64_t hm = J[w] & ~I[w], pm = I[w] & ~J[w];
        while (hm) { int b = __builtin_ctzll(hm); e->holes[nh++] = 64 * w + b; hm &= hm - 1; }
        while (pm) { int b = __builtin_ctzll(pm); e->parts[np++] = 64 * w + b; pm &= pm - 1; }
    }
    if (e->degree == 1) {
        e->phase = (popc_between(J, nw, e->holes[0], e->parts[0]) & 1) ? -1 : 1;
        return;
    }
    /* double: a+_p1 a+_p2 a_h2 a_h1 = (a+_p1 a_h1)(a+_p2 a_h2); apply h2->p2 to J
       first, then h1->p1 to the intermediate string */
    uint64_t Jm[2 * ORC_MAXW];
    memcpy(Jm, J, sizeof(uint64_t) * nw);
    int s2 = popc_between(J, nw, e->holes[1], e->parts[1]);
    Jm[e->holes[1] / 64] &= ~(1ull << (e->holes[1] % 64));
    Jm[e->parts[1] / 64] |= (1ull << (e->parts[1] % 64));
    int s1 = popc_between(Jm, nw, e->holes[0], e->parts[0]);
    e->phase = ((s1 + s2) & 1) ? -1 : 1;
}

/* ------------------------------------------------------------------------ */
/* symbolic Slater-Condon (Eq. 6) over an orbital space of `norb` spatial     */
/* orbitals per spin, packed in `wps` words per spin.                         */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t label; double coef; } orc_sym;

static uint64_t lab2(int p, int q, int r, int s) {
    /* canonical 8-fold representative: p>=q, r>=s, (p,q) >= (r,s) */
    if (p < q) { int t = p; p = q; q = t; }
    if (r < s) { int t = r; r = s; s = t; }
    if (p < r || (p == r && q < s)) { int t; t = p; p = r; r = t; t = q; q = s; s = t; }
    return (uint64_t)p | ((uint64_t)q << 16) | ((uint64_t)r << 32) | ((uint64_t)s << 48);
}
static uint64_t lab1(int p, int q) {
    if (p < q) { int t = p; p = q; q = t; }
    return (uint64_t)p | ((uint64_t)q << 16) | ((uint64_t)ORC_ONE_E << 32) | ((uint64_t)ORC_ONE_E << 48);
}

/* Emit the symbols of <I|H|J>.  Returns the number written (<= cap). */
static int orc_symbols(int wps, const uint64_t *I, const uint64_t *J, orc_sym *out, int cap) {
    const int nw = 2 * wps, sb = 64 * wps; /* bits per spin string */
    orc_exc e;
    orc_excitation(nw, I, J, &e);
    int n = 0;
#define EMIT(L, C) do { if (n < cap) { out[n].label = (L); out[n].coef = (C); } ++n; } while (0)
    if (e.degree > 2) return 0;
    if (e.degree == 0) {
        int occ[512], no = 0;
        for (int w = 0; w < nw; ++w) { uint64_t x = I[w]; while (x) { occ[no++] = 64 * w + __builtin_ctzll(x); x &= x - 1; } }
        for (int a = 0; a < no; ++a) {
            int pa = occ[a] % sb;
            EMIT(lab1(pa, pa), 1.0);
        }
        for (int a = 0; a < no; ++a)
            for (int b = a + 1; b < no; ++b) {
                int pa = occ[a] % sb, pb = occ[b] % sb;
                EMIT(lab2(pa, pa, pb, pb), 1.0);
                if (occ[a] / sb == occ[b] / sb) EMIT(lab2(pa, pb, pb, pa), -1.0);
            }
        return n;
    }
    if (e.degree == 1) {
        int h = e.holes[0], p = e.parts[0];
        int hs = h / sb, ho = h % sb, po = p % sb;
        double ph = (double)e.phase;
        EMIT(lab1(po, ho), ph);
        for (int w = 0; w < nw; ++w) {
            uint64_t x = I[w] & J[w];
            while (x) {
                int k = 64 * w + __builtin_ctzll(x); x &= x - 1;
                int ko = k % sb;
                EMIT(lab2(po, ho, ko, ko), ph);
                if (k / sb == hs) EMIT(lab2(po, ko, ko, ho), -ph);
            }
        }
        return n;
    }
    /* degree 2 */
    {
        int h1 = e.holes[0], h2 = e.holes[1], p1 = e.parts[0], p2 = e.parts[1];
        int s_h1 = h1 / sb, s_h2 = h2 / sb, s_p1 = p1 / sb, s_p2 = p2 / sb;
        double ph = (double)e.phase;
        if (s_p1 == s_h1 && s_p2 == s_h2) EMIT(lab2(p1 % sb, h1 % sb, p2 % sb, h2 % sb), ph);
        if (s_p1 == s_h2 && s_p2 == s_h1) EMIT(lab2(p1 % sb, h2 % sb, p2 % sb, h1 % sb), -ph);
        return n;
    }
#undef EMIT
}

/* X(I) with placeholder substitution: orbital index `ph_bra` -> global
   continuum orbital jb, `ph_ket` -> jk; other indices are target orbitals. */
static double orc_X(const orc_problem *P, uint64_t label, int ph_bra, int jb, int ph_ket, int jk) {
    int idx[4];
    for (int k = 0; k < 4; ++k) idx[k] = (int)((label >> (16 * k)) & 0xFFFFu);
    if (idx[2] == (int)ORC_ONE_E) {
        int p = idx[0] == ph_bra ? jb : (idx[0] == ph_ket ? jk : idx[0]);
        int q = idx[1] == ph_bra ? jb : (idx[1] == ph_ket ? jk : idx[1]);
        return orc_one(P, p, q);
    }
    for (int k = 0; k < 4; ++k) {
        if (idx[k] == ph_bra) idx[k] = jb;
        else if (idx[k] == ph_ket) idx[k] = jk;
    }
    return orc_two(P, idx[0], idx[1], idx[2], idx[3]);
}

/* ------------------------------------------------------------------------ */
/* numeric Slater-Condon for two target-space determinants (classes 2, 8 and */
/* the target Hamiltonian)                                                    */
/* ------------------------------------------------------------------------ */

double orc_hij(const orc_problem *P, const uint64_t *I, const uint64_t *J) {
    orc_sym buf[4096];
    int n = orc_symbols(P->W, I, J, buf, 4096);
    double v = 0.0;
    for (int k = 0; k < n && k < 4096; ++k) v += buf[k].coef * orc_X(P, buf[k].label, -1, 0, -1, 0);
    return v;
}

/* API for the excitation-classification parity tests.  out[0] degree,
   out[1..2] holes, out[3..4] particles, out[5] phase.  Degree > 2 leaves the
   rest undefined (holes/particles -1, phase +1). */
int orc_excitation_api(int W, const uint64_t *I, const uint64_t *J, int32_t *out) {
    orc_exc e;
    orc_excitation(2 * W, I, J, &e);
    out[0] = e.degree;
    out[1] = e.holes[0]; out[2] = e.holes[1];
    out[3] = e.parts[0]; out[4] = e.parts[1];
    out[5] = e.degree <= 2 ? e.phase : 1;
    return e.degree;
}

/* ------------------------------------------------------------------------ */
/* extended strings: target orbitals plus two placeholder orbitals n_to       */
/* (bra continuum) and n_to+1 (ket continuum) in each spin string.            */
/* ------------------------------------------------------------------------ */

static int ext_words(const orc_problem *P) { return (P->n_to + 2 + 63) / 64; }

static void extend(const orc_problem *P, const uint64_t *D, int place, int spin, uint64_t *X) {
    const int W = P->W, We = ext_words(P);
    memset(X, 0, sizeof(uint64_t) * 2 * We);
    for (int s = 0; s < 2; ++s)
        for (int w = 0; w < W; ++w) X[s * We + w] = D[s * W + w];
    if (place >= 0) X[spin * We + place / 64] |= 1ull << (place % 64);
}

/* T x L2 classification record in the same form the CUDA classifier
   reports: the bra is D_m plus a continuum electron above every target
   orbital of spin cont_spin.  out[0] degree (of the (N+1)-electron pair),
   out[1..2] target holes (bit positions in the W-word layout, in chi only),
   out[3] target particle (in D_m only), out[4] phase.  Returns degree. */
int orc_excitation_tl2(const orc_problem *P, const uint64_t *D, const uint64_t *chi, int32_t *out) {
    uint64_t I[2 * ORC_MAXW], J[2 * ORC_MAXW];
    const int We = ext_words(P), W = P->W;
    extend(P, D, P->n_to, P->cont_spin, I);
    extend(P, chi, -1, 0, J);
    orc_exc e;
    orc_excitation(2 * We, I, J, &e);
    out[0] = e.degree;
    out[1] = out[2] = out[3] = -1;
    out[4] = 1;
    if (e.degree > 2) return e.degree;
    int nh = 0;
    for (int k = 0; k < e.degree; ++k) {
        int b = e.holes[k], s = b / (64 * We), o = b % (64 * We);
        out[1 + nh++] = s * 64 * W + o;
    }
    for (int k = 0; k < e.degree; ++k) {
        int b = e.parts[k], s = b / (64 * We), o = b % (64 * We);
        if (o == P->n_to) continue; /* the continuum electron */
        out[3] = s * 64 * W + o;
    }
    out[4] = e.phase;
    return e.degree;
}

/* ------------------------------------------------------------------------ */
/* label -> coefficient block map (open addressing)                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t *keys;
    int32_t *slot;
    int64_t cap;      /* hash capacity (power of two) */
    int64_t n;        /* labels stored */
    int64_t bsz;      /* doubles per block */
    double *blocks;   /* n * bsz */
    int64_t bcap;     /* allocated blocks */
} orc_map;

static void map_init(orc_map *m, int64_t bsz) {
    m->cap = 1024; m->n = 0; m->bsz = bsz; m->bcap = 64;
    m->keys = (uint64_t *)malloc(sizeof(uint64_t) * m->cap);
    m->slot = (int32_t *)malloc(sizeof(int32_t) * m->cap);
    for (int64_t i = 0; i < m->cap; ++i) m->slot[i] = -1;
    m->blocks = (double *)calloc((size_t)(m->bcap * bsz), sizeof(double));
}
static void map_free(orc_map *m) { free(m->keys); free(m->slot); free(m->blocks); }
/* Empty the map, keeping its storage. */
static void map_reset(orc_map *m) {
    memset(m->blocks, 0, sizeof(double) * (size_t)(m->n * m->bsz));
    for (int64_t i = 0; i < m->cap; ++i) m->slot[i] = -1;
    m->n = 0;
}
static uint64_t hmix(uint64_t x) { x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull; x ^= x >> 33; return x; }

static double *map_get(orc_map *m, uint64_t key) {
    if (2 * (m->n + 1) > m->cap) {
        int64_t nc = m->cap * 2;
        uint64_t *nk = (uint64_t *)malloc(sizeof(uint64_t) * nc);
        int32_t *ns = (int32_t *)malloc(sizeof(int32_t) * nc);
        for (int64_t i = 0; i < nc; ++i) ns[i] = -1;
        for (int64_t i = 0; i < m->cap; ++i)
            if (m->slot[i] >= 0) {
                int64_t h = (int64_t)(hmix(m->keys[i]) & (uint64_t)(nc - 1));
                while (ns[h] >= 0) h = (h + 1) & (nc - 1);
                nk[h] = m->keys[i]; ns[h] = m->slot[i];
            }
        free(m->keys); free(m->slot); m->keys = nk; m->slot = ns; m->cap = nc;
    }
    int64_t h = (int64_t)(hmix(key) & (uint64_t)(m->cap - 1));
    while (m->slot[h] >= 0) {
        if (m->keys[h] == key) return m->blocks + (int64_t)m->slot[h] * m->bsz;
        h = (h + 1) & (m->cap - 1);
    }
    if (m->n == m->bcap) {
        int64_t nb = m->bcap * 2;
        m->blocks = (double *)realloc(m->blocks, sizeof(double) * (size_t)(nb * m->bsz));
        memset(m->blocks + m->bcap * m->bsz, 0, sizeof(double) * (size_t)((nb - m->bcap) * m->bsz));
        m->bcap = nb;
    }
    m->keys[h] = key; m->slot[h] = (int32_t)m->n;
    return m->blocks + (m->n++) * m->bsz;
}

/* ------------------------------------------------------------------------ */
/* continuum-continuum classes 1,3,5,6,7: contraction (Eq. 8)                */
/* ------------------------------------------------------------------------ */

typedef struct {
    const orc_problem *P;
    int g, gp, ns, nsp;
    orc_map same;   /* same continuum orbital prototype, labels with placeholder */
    orc_map diff;   /* different continuum orbitals prototype */
    double *K0;     /* j-independent part of the same-orbital prototype [n][n'] */
    /* the same sums over |c_mn c_m'n' C| (|c c C X| for K0): the magnitudes of
       the terms the contraction (Eq. 8) adds, for the full condition scale */
    orc_map same_abs, diff_abs;
    double *K0abs;
    int with_abs;   /* 0: the magnitudes were not accumulated */
} orc_cc;

/* Merge map b into map a (blocks added label by label). */
static void map_merge(orc_map *a, const orc_map *b) {
    for (int64_t i = 0; i < b->cap; ++i) {
        const int s = b->slot[i];
        if (s < 0) continue;
        double *dst = map_get(a, b->keys[i]);
        const double *src = b->blocks + (int64_t)s * b->bsz;
        for (int64_t t = 0; t < a->bsz; ++t) dst[t] += src[t];
    }
}

orc_cc *orc_cc_contract_ex(const orc_problem *P, int g, int gp, int with_abs) {
    orc_cc *c = (orc_cc *)calloc(1, sizeof(orc_cc));
    c->with_abs = with_abs;
    c->P = P; c->g = g; c->gp = gp;
    c->ns = P->g_nstate[g]; c->nsp = P->g_nstate[gp];
    const int ns = c->ns, nsp = c->nsp, bsz = ns * nsp;
    map_init(&c->same, bsz);
    map_init(&c->diff, bsz);
    map_init(&c->same_abs, bsz);
    map_init(&c->diff_abs, bsz);
    c->K0 = (double *)calloc((size_t)bsz, sizeof(double));
    c->K0abs = (double *)calloc((size_t)bsz, sizeof(double));
    const int W = P->W, We = ext_words(P), ph = P->n_to, phk = P->n_to + 1, sc = P->cont_spin;
    const uint64_t *Dg = P->g_dets[g], *Dgp = P->g_dets[gp];
    const double *Cg = P->g_ci[g], *Cgp = P->g_ci[gp];
    /* bra determinants are split into ORC_CHUNKS fixed chunks whatever the
       thread count; a thread contracts a chunk into its own maps (the Eq. 8
       sums over the chunk's determinants in order) and merges them into the
       result in chunk order, so the sums, and the label order of the merged
       maps, do not depend on the number of threads */
    const int ndet_g = P->g_ndet[g];
    const int nchunk = ndet_g < ORC_CHUNKS ? ndet_g : ORC_CHUNKS;
#pragma omp parallel
    {
        orc_map same, diff, same_a, diff_a;
        map_init(&same, bsz);
        map_init(&diff, bsz);
        map_init(&same_a, bsz);
        map_init(&diff_a, bsz);
        double *K0 = (double *)calloc((size_t)bsz, sizeof(double));
        double *K0a = (double *)calloc((size_t)bsz, sizeof(double));
        orc_sym *buf = (orc_sym *)malloc(sizeof(orc_sym) * 8192);
        double *cc = (double *)malloc(sizeof(double) * bsz);
        uint64_t I[2 * ORC_MAXW], J[2 * ORC_MAXW];
#pragma omp for ordered schedule(dynamic, 1)
        for (int ch = 0; ch < nchunk; ++ch) {
            const int m0 = (int)((int64_t)ndet_g * ch / nchunk), m1 = (int)((int64_t)ndet_g * (ch + 1) / nchunk);
            map_reset(&same);
            map_reset(&diff);
            map_reset(&same_a);
            map_reset(&diff_a);
            memset(K0, 0, sizeof(double) * (size_t)bsz);
            memset(K0a, 0, sizeof(double) * (size_t)bsz);
            for (int m = m0; m < m1; ++m) {
                const uint64_t *Dm = Dg + (int64_t)m * 2 * W;
                for (int mp = 0; mp < P->g_ndet[gp]; ++mp) {
                    const uint64_t *Dmp = Dgp + (int64_t)mp * 2 * W;
                    int nd = 0;
                    for (int w = 0; w < 2 * W; ++w) nd += popc64(Dm[w] ^ Dmp[w]);
                    if (nd > 4) continue;
                    for (int a = 0; a < ns; ++a)
                        for (int b = 0; b < nsp; ++b)
                            cc[a * nsp + b] = Cg[(int64_t)m * ns + a] * Cgp[(int64_t)mp * nsp + b];
                    /* prototype 1: the same continuum orbital in bra and ket */
                    extend(P, Dm, ph, sc, I);
                    extend(P, Dmp, ph, sc, J);
                    int n = orc_symbols(We, I, J, buf, 8192);
                    for (int k = 0; k < n; ++k) {
                        uint64_t L = buf[k].label;
                        int has = 0;
                        for (int s2 = 0; s2 < 4; ++s2) has |= (int)(((L >> (16 * s2)) & 0xFFFFu) == (uint64_t)ph);
                        if (!has) {
                            if (P->g_energy) continue;   /* replaced by the target energies below */
                            double x = buf[k].coef * orc_X(P, L, -1, 0, -1, 0);
                            for (int t = 0; t < bsz; ++t) K0[t] += cc[t] * x;
                            if (with_abs) for (int t = 0; t < bsz; ++t) K0a[t] += fabs(cc[t] * x);
                        } else {
                            double *blk = map_get(&same, L);
                            for (int t = 0; t < bsz; ++t) blk[t] += cc[t] * buf[k].coef;
                            if (with_abs) {
                                blk = map_get(&same_a, L);
                                for (int t = 0; t < bsz; ++t) blk[t] += fabs(cc[t] * buf[k].coef);
                            }
                        }
                    }
                    if (nd == 0 && P->e_core != 0.0 && !P->g_energy) {
                        for (int t = 0; t < bsz; ++t) K0[t] += cc[t] * P->e_core;
                        if (with_abs) for (int t = 0; t < bsz; ++t) K0a[t] += fabs(cc[t] * P->e_core);
                    }
                    /* prototype 2: different continuum orbitals (j in bra, j' in ket) */
                    if (nd <= 2) {
                        extend(P, Dm, ph, sc, I);
                        extend(P, Dmp, phk, sc, J);
                        n = orc_symbols(We, I, J, buf, 8192);
                        for (int k = 0; k < n; ++k) {
                            double *blk = map_get(&diff, buf[k].label);
                            for (int t = 0; t < bsz; ++t) blk[t] += cc[t] * buf[k].coef;
                            if (with_abs) {
                                blk = map_get(&diff_a, buf[k].label);
                                for (int t = 0; t < bsz; ++t) blk[t] += fabs(cc[t] * buf[k].coef);
                            }
                        }
                    }
                }
            }
#pragma omp ordered
            {
                map_merge(&c->same, &same);
                map_merge(&c->diff, &diff);
                map_merge(&c->same_abs, &same_a);
                map_merge(&c->diff_abs, &diff_a);
                for (int t = 0; t < bsz; ++t) c->K0[t] += K0[t];
                for (int t = 0; t < bsz; ++t) c->K0abs[t] += K0a[t];
            }
        }
        map_free(&same);
        map_free(&diff);
        map_free(&same_a);
        map_free(&diff_a);
        free(K0);
        free(K0a);
        free(buf);
        free(cc);
    }
    if (P->g_energy) {
        /* the target states are eigenstates of H^N + e_core: their target-only
           part is delta_gg' delta_nn' E_n (Section 3.1) */
        for (int a = 0; a < ns; ++a)
            for (int b = 0; b < nsp; ++b) {
                c->K0[a * nsp + b] = (g == gp && a == b) ? P->g_energy[g][a] : 0.0;
                c->K0abs[a * nsp + b] = fabs(c->K0[a * nsp + b]);
            }
    }
    return c;
}

orc_cc *orc_cc_contract(const orc_problem *P, int g, int gp) { return orc_cc_contract_ex(P, g, gp, 1); }

void orc_cc_free(orc_cc *c) {
    map_free(&c->same); map_free(&c->diff); map_free(&c->same_abs); map_free(&c->diff_abs);
    free(c->K0); free(c->K0abs); free(c);
}

int64_t orc_cc_nlabels(const orc_cc *c, int which) { return which ? c->diff.n : c->same.n; }

/* Eq. 7: one contracted element <g n j | H | g' n' j'>, j and j' are
   continuum indices (0-based within the continuum). */
double orc_cc_element(const orc_cc *c, int n, int j, int np, int jp) {
    const orc_problem *P = c->P;
    const int ph = P->n_to, phk = P->n_to + 1, t = n * c->nsp + np;
    const int jg = P->n_to + j, jpg = P->n_to + jp;
    double v = 0.0;
    if (j == jp) {
        v = c->K0[t];
        for (int64_t i = 0; i < c->same.cap; ++i) {
            int s = c->same.slot[i];
            if (s < 0) continue;
            double d = c->same.blocks[(int64_t)s * c->same.bsz + t];
            if (d != 0.0) v += d * orc_X(P, c->same.keys[i], ph, jg, -1, 0);
        }
    } else {
        for (int64_t i = 0; i < c->diff.cap; ++i) {
            int s = c->diff.slot[i];
            if (s < 0) continue;
            double d = c->diff.blocks[(int64_t)s * c->diff.bsz + t];
            if (d != 0.0) v += d * orc_X(P, c->diff.keys[i], ph, jg, phk, jpg);
        }
    }
    return v;
}

/* Expand a whole group-pair block into dense H (full symmetric storage,
   leading dimension ld), rows/cols offset by the groups' positions. */
void orc_cc_expand(const orc_cc *c, double *H, int64_t ld, int64_t row0, int64_t col0) {
    const orc_problem *P = c->P;
    const int cfg = P->g_cfirst[c->g], cng = P->g_ccount[c->g];
    const int cfp = P->g_cfirst[c->gp], cnp = P->g_ccount[c->gp];
    /* flatten the maps for the inner loop */
    const int64_t ns_ = c->same.n, nd_ = c->diff.n;
    uint64_t *ks = (uint64_t *)malloc(sizeof(uint64_t) * (ns_ + 1));
    uint64_t *kd = (uint64_t *)malloc(sizeof(uint64_t) * (nd_ + 1));
    for (int64_t i = 0; i < c->same.cap; ++i) if (c->same.slot[i] >= 0) ks[c->same.slot[i]] = c->same.keys[i];
    for (int64_t i = 0; i < c->diff.cap; ++i) if (c->diff.slot[i] >= 0) kd[c->diff.slot[i]] = c->diff.keys[i];
    const int ph = P->n_to, phk = P->n_to + 1, bsz = c->ns * c->nsp;
#pragma omp parallel for schedule(dynamic, 1)
    for (int jj = 0; jj < cng; ++jj) {
        double *xs = (double *)malloc(sizeof(double) * (ns_ + 1));
        double *xd = (double *)malloc(sizeof(double) * (nd_ + 1));
        const int j = cfg + jj;
        for (int jjp = 0; jjp < cnp; ++jjp) {
            const int jp = cfp + jjp;
            const int same = (j == jp);
            if (same) for (int64_t i = 0; i < ns_; ++i) xs[i] = orc_X(P, ks[i], ph, P->n_to + j, -1, 0);
            else for (int64_t i = 0; i < nd_; ++i) xd[i] = orc_X(P, kd[i], ph, P->n_to + j, phk, P->n_to + jp);
            for (int n = 0; n < c->ns; ++n)
                for (int np = 0; np < c->nsp; ++np) {
                    const int t = n * c->nsp + np;
                    int64_t r = row0 + (int64_t)n * cng + jj, cl = col0 + (int64_t)np * cnp + jjp;
                    if (c->g == c->gp && r < cl) continue; /* lower triangle, then mirror */
                    double v = 0.0;
                    if (same) {
                        v = c->K0[t];
                        for (int64_t i = 0; i < ns_; ++i) v += c->same.blocks[i * bsz + t] * xs[i];
                    } else {
                        for (int64_t i = 0; i < nd_; ++i) v += c->diff.blocks[i * bsz + t] * xd[i];
                    }
                    H[r * ld + cl] = v;
                    H[cl * ld + r] = v;
                }
        }
        free(xs); free(xd);
    }
    free(ks); free(kd);
}

/* ------------------------------------------------------------------------ */
/* class 4: continuum x L2 (Eq. 5)                                           */
/* ------------------------------------------------------------------------ */

/* One L2 row: out[(g, n, j)] = <Psi_{g n j}|H|chi_l> for every group, in the
   contracted basis order.  Prototype (one continuum placeholder) per pair
   (m, l), contraction over m, expansion over j. */
void orc_class4_row(const orc_problem *P, int l, double *out) {
    const int W = P->W, We = ext_words(P), ph = P->n_to, sc = P->cont_spin;
    const uint64_t *chi = P->l2 + (int64_t)l * 2 * W;
    uint64_t I[2 * ORC_MAXW], J[2 * ORC_MAXW];
    orc_sym buf[4096];
    int64_t off = 0;
    extend(P, chi, -1, 0, J);
    for (int g = 0; g < P->n_groups; ++g) {
        const int ns = P->g_nstate[g], cf = P->g_cfirst[g], cn = P->g_ccount[g];
        orc_map A;
        map_init(&A, ns);
        const uint64_t *Dg = P->g_dets[g];
        const double *Cg = P->g_ci[g];
        for (int m = 0; m < P->g_ndet[g]; ++m) {
            const uint64_t *Dm = Dg + (int64_t)m * 2 * W;
            /* electrons of D_m missing from chi: d = 0 or 1 contribute */
            int d = 0;
            for (int w = 0; w < 2 * W; ++w) d += popc64(Dm[w] & ~chi[w]);
            if (d > 1) continue;
            extend(P, Dm, ph, sc, I);
            int n = orc_symbols(We, I, J, buf, 4096);
            for (int k = 0; k < n; ++k) {
                double *blk = map_get(&A, buf[k].label);
                for (int a = 0; a < ns; ++a) blk[a] += Cg[(int64_t)m * ns + a] * buf[k].coef;
            }
        }
        for (int jj = 0; jj < cn; ++jj) {
            const int jg = P->n_to + cf + jj;
            for (int a = 0; a < ns; ++a) out[off + (int64_t)a * cn + jj] = 0.0;
            for (int64_t i = 0; i < A.cap; ++i) {
                int s = A.slot[i];
                if (s < 0) continue;
                double x = orc_X(P, A.keys[i], ph, jg, -1, 0);
                for (int a = 0; a < ns; ++a) out[off + (int64_t)a * cn + jj] += A.blocks[(int64_t)s * ns + a] * x;
            }
        }
        map_free(&A);
        off += (int64_t)ns * cn;
    }
}

/* ------------------------------------------------------------------------ */
/* classes 2 and 8: L2 x L2                                                  */
/* ------------------------------------------------------------------------ */

double orc_l2_element(const orc_problem *P, int a, int b) {
    const int W = P->W;
    double v = orc_hij(P, P->l2 + (int64_t)a * 2 * W, P->l2 + (int64_t)b * 2 * W);
    if (a == b) v += P->e_core;
    return v;
}

/* ------------------------------------------------------------------------ */
/* whole matrix, dense, full symmetric storage (small problems)              */
/* ------------------------------------------------------------------------ */

int64_t orc_contracted_dim(const orc_problem *P) {
    int64_t d = 0;
    for (int g = 0; g < P->n_groups; ++g) d += (int64_t)P->g_nstate[g] * P->g_ccount[g];
    return d;
}

void orc_build_dense(const orc_problem *P, double *H) {
    const int64_t Dc = orc_contracted_dim(P), dim = Dc + P->n_l2;
    memset(H, 0, sizeof(double) * (size_t)(dim * dim));
    int64_t off_g = 0;
    for (int g = 0; g < P->n_groups; ++g) {
        int64_t off_gp = 0;
        for (int gp = 0; gp <= g; ++gp) {
            orc_cc *c = orc_cc_contract(P, g, gp);
            orc_cc_expand(c, H, dim, off_g, off_gp);
            orc_cc_free(c);
            off_gp += (int64_t)P->g_nstate[gp] * P->g_ccount[gp];
        }
        off_g += (int64_t)P->g_nstate[g] * P->g_ccount[g];
    }
#pragma omp parallel
    {
        double *row = (double *)malloc(sizeof(double) * (size_t)(Dc + 1));
#pragma omp for schedule(dynamic, 4)
        for (int l = 0; l < P->n_l2; ++l) {
            orc_class4_row(P, l, row);
            for (int64_t c = 0; c < Dc; ++c) {
                H[(Dc + l) * dim + c] = row[c];
                H[c * dim + Dc + l] = row[c];
            }
        }
        free(row);
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int a = 0; a < P->n_l2; ++a)
        for (int b = 0; b <= a; ++b) {
            double v = orc_l2_element(P, a, b);
            H[(Dc + a) * dim + Dc + b] = v;
            H[(Dc + b) * dim + Dc + a] = v;
        }
}

/* L2 block only: CSR of the full symmetric L2 x L2 block (|value| > 0 means a
   pair within double excitation; exact zeros from cancellation are kept).  The
   first call with vals == NULL returns nnz in *nnz and fills row_ptr. */
void orc_l2_csr(const orc_problem *P, int64_t *row_ptr, int32_t *cols, double *vals) {
    const int W = P->W, nl = P->n_l2;
    if (!vals) {
        row_ptr[0] = 0;
#pragma omp parallel for schedule(dynamic, 64)
        for (int a = 0; a < nl; ++a) {
            int64_t c = 0;
            for (int b = 0; b < nl; ++b) {
                int nd = 0;
                for (int w = 0; w < 2 * W; ++w) nd += popc64(P->l2[(int64_t)a * 2 * W + w] ^ P->l2[(int64_t)b * 2 * W + w]);
                c += (nd <= 4);
            }
            row_ptr[a + 1] = c;
        }
        for (int a = 0; a < nl; ++a) row_ptr[a + 1] += row_ptr[a];
        return;
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int a = 0; a < nl; ++a) {
        int64_t k = row_ptr[a];
        for (int b = 0; b < nl; ++b) {
            int nd = 0;
            for (int w = 0; w < 2 * W; ++w) nd += popc64(P->l2[(int64_t)a * 2 * W + w] ^ P->l2[(int64_t)b * 2 * W + w]);
            if (nd <= 4) { cols[k] = b; vals[k] = orc_l2_element(P, a, b); ++k; }
        }
    }
}

/* Dense rows [a0, a1) of the L2 x L2 block (row-major, n_l2 columns). */
void orc_l2_rows(const orc_problem *P, int a0, int a1, double *out) {
    const int nl = P->n_l2;
#pragma omp parallel for schedule(dynamic, 4)
    for (int a = a0; a < a1; ++a) {
        const int W = P->W;
        for (int b = 0; b < nl; ++b) {
            int nd = 0;
            for (int w = 0; w < 2 * W; ++w) nd += popc64(P->l2[(int64_t)a * 2 * W + w] ^ P->l2[(int64_t)b * 2 * W + w]);
            out[(int64_t)(a - a0) * nl + b] = nd <= 4 ? orc_l2_element(P, a, b) : 0.0;
        }
    }
}

/* Class-4 rows [l0, l1) into out[(l - l0) * Dc + c]. */
void orc_class4_rows(const orc_problem *P, int l0, int l1, double *out) {
    const int64_t Dc = orc_contracted_dim(P);
#pragma omp parallel for schedule(dynamic, 4)
    for (int l = l0; l < l1; ++l) orc_class4_row(P, l, out + (int64_t)(l - l0) * Dc);
}

/* Condition scale of a contracted continuum element: sum over labels of
   |D^b X(I^b)| (Eq. 7 with absolute values).  This is the natural size of the
   rounding error of any finite-precision evaluation of the sum. */
double orc_cc_element_abs(const orc_cc *c, int n, int j, int np, int jp) {
    const orc_problem *P = c->P;
    const int ph = P->n_to, phk = P->n_to + 1, t = n * c->nsp + np;
    const int jg = P->n_to + j, jpg = P->n_to + jp;
    double v = 0.0;
    if (j == jp) {
        v = fabs(c->K0[t]);
        for (int64_t i = 0; i < c->same.cap; ++i) {
            int s = c->same.slot[i];
            if (s < 0) continue;
            v += fabs(c->same.blocks[(int64_t)s * c->same.bsz + t] * orc_X(P, c->same.keys[i], ph, jg, -1, 0));
        }
    } else {
        for (int64_t i = 0; i < c->diff.cap; ++i) {
            int s = c->diff.slot[i];
            if (s < 0) continue;
            v += fabs(c->diff.blocks[(int64_t)s * c->diff.bsz + t] * orc_X(P, c->diff.keys[i], ph, jg, phk, jpg));
        }
    }
    return v;
}

/* The same for a whole group-pair block, written like orc_cc_expand. */
void orc_cc_expand_abs(const orc_cc *c, double *H, int64_t ld, int64_t row0, int64_t col0) {
    const orc_problem *P = c->P;
    const int cfg = P->g_cfirst[c->g], cng = P->g_ccount[c->g];
    const int cfp = P->g_cfirst[c->gp], cnp = P->g_ccount[c->gp];
#pragma omp parallel for schedule(dynamic, 1)
    for (int jj = 0; jj < cng; ++jj)
        for (int jjp = 0; jjp < cnp; ++jjp)
            for (int n = 0; n < c->ns; ++n)
                for (int np = 0; np < c->nsp; ++np) {
                    int64_t r = row0 + (int64_t)n * cng + jj, cl = col0 + (int64_t)np * cnp + jjp;
                    if (c->g == c->gp && r < cl) continue;
                    double v = orc_cc_element_abs(c, n, cfg + jj, np, cfp + jjp);
                    H[r * ld + cl] = v;
                    H[cl * ld + r] = v;
                }
}

/* Expansion (Eq. 7) of the rows jj in [jj0, jj1) of a group-pair block only,
   for every state pair (a bounded sample of orc_cc_expand): the integrals of
   every label are looked up once per (j, j'), then used for all (n, n'). */
void orc_cc_expand_rows(const orc_cc *c, double *out, int jj0, int jj1) {
    const orc_problem *P = c->P;
    const int cfg = P->g_cfirst[c->g];
    const int cfp = P->g_cfirst[c->gp], cnp = P->g_ccount[c->gp];
    const int nr = jj1 - jj0, bsz = c->ns * c->nsp;
    const int64_t ns_ = c->same.n, nd_ = c->diff.n;
    uint64_t *ks = (uint64_t *)malloc(sizeof(uint64_t) * (ns_ + 1));
    uint64_t *kd = (uint64_t *)malloc(sizeof(uint64_t) * (nd_ + 1));
    for (int64_t i = 0; i < c->same.cap; ++i) if (c->same.slot[i] >= 0) ks[c->same.slot[i]] = c->same.keys[i];
    for (int64_t i = 0; i < c->diff.cap; ++i) if (c->diff.slot[i] >= 0) kd[c->diff.slot[i]] = c->diff.keys[i];
    const int ph = P->n_to, phk = P->n_to + 1;
#pragma omp parallel
    {
        double *xs = (double *)malloc(sizeof(double) * (ns_ + 1));
        double *xd = (double *)malloc(sizeof(double) * (nd_ + 1));
#pragma omp for collapse(2) schedule(dynamic, 4)
        for (int r = 0; r < nr; ++r)
            for (int jjp = 0; jjp < cnp; ++jjp) {
                const int j = cfg + jj0 + r, jp = cfp + jjp;
                const int same = (j == jp);
                if (same) for (int64_t i = 0; i < ns_; ++i) xs[i] = orc_X(P, ks[i], ph, P->n_to + j, -1, 0);
                else for (int64_t i = 0; i < nd_; ++i) xd[i] = orc_X(P, kd[i], ph, P->n_to + j, phk, P->n_to + jp);
                double *o = out + ((int64_t)r * cnp + jjp) * bsz;
                for (int t = 0; t < bsz; ++t) {
                    double v = 0.0;
                    if (same) {
                        v = c->K0[t];
                        for (int64_t i = 0; i < ns_; ++i) v += c->same.blocks[i * bsz + t] * xs[i];
                    } else {
                        for (int64_t i = 0; i < nd_; ++i) v += c->diff.blocks[i * bsz + t] * xd[i];
                    }
                    o[t] = v;
                }
            }
        free(xs);
        free(xd);
    }
    free(ks);
    free(kd);
}

/* Condition scale of the class-4 row l (Eq. 5 with absolute values): for
   every contracted column (g, n, j), sum over the target determinants m and
   the labels of their prototype against chi_l of |c_mn C X(I)|, the sum of
   the magnitudes of the terms that any evaluation order adds. */
void orc_class4_row_abs(const orc_problem *P, int l, double *out) {
    const int W = P->W, We = ext_words(P), ph = P->n_to, sc = P->cont_spin;
    const uint64_t *chi = P->l2 + (int64_t)l * 2 * W;
    uint64_t I[2 * ORC_MAXW], J[2 * ORC_MAXW];
    orc_sym buf[4096];
    int64_t off = 0;
    extend(P, chi, -1, 0, J);
    for (int g = 0; g < P->n_groups; ++g) {
        const int ns = P->g_nstate[g], cf = P->g_cfirst[g], cn = P->g_ccount[g];
        const uint64_t *Dg = P->g_dets[g];
        const double *Cg = P->g_ci[g];
        for (int64_t t = 0; t < (int64_t)ns * cn; ++t) out[off + t] = 0.0;
        for (int m = 0; m < P->g_ndet[g]; ++m) {
            const uint64_t *Dm = Dg + (int64_t)m * 2 * W;
            int d = 0;
            for (int w = 0; w < 2 * W; ++w) d += popc64(Dm[w] & ~chi[w]);
            if (d > 1) continue;
            extend(P, Dm, ph, sc, I);
            int n = orc_symbols(We, I, J, buf, 4096);
            for (int jj = 0; jj < cn; ++jj) {
                const int jg = P->n_to + cf + jj;
                double s = 0.0;
                for (int k = 0; k < n; ++k) s += fabs(buf[k].coef * orc_X(P, buf[k].label, ph, jg, -1, 0));
                for (int a = 0; a < ns; ++a) out[off + (int64_t)a * cn + jj] += fabs(Cg[(int64_t)m * ns + a]) * s;
            }
        }
        off += (int64_t)ns * cn;
    }
}

/* Condition scale of an L2-L2 element: sum of |C X(I)| over its symbols
   (plus |e_core| on the diagonal). */
double orc_l2_element_abs(const orc_problem *P, int a, int b) {
    const int W = P->W;
    orc_sym buf[4096];
    int n = orc_symbols(W, P->l2 + (int64_t)a * 2 * W, P->l2 + (int64_t)b * 2 * W, buf, 4096);
    double v = 0.0;
    for (int k = 0; k < n && k < 4096; ++k) v += fabs(buf[k].coef * orc_X(P, buf[k].label, -1, 0, -1, 0));
    if (a == b) v += fabs(P->e_core);
    return v;
}

/* Condition scales of the dense rows [a0, a1) of the L2 x L2 block. */
void orc_l2_rows_abs(const orc_problem *P, int a0, int a1, double *out) {
    const int nl = P->n_l2, W = P->W;
#pragma omp parallel for schedule(dynamic, 4)
    for (int a = a0; a < a1; ++a)
        for (int b = 0; b < nl; ++b) {
            int nd = 0;
            for (int w = 0; w < 2 * W; ++w) nd += popc64(P->l2[(int64_t)a * 2 * W + w] ^ P->l2[(int64_t)b * 2 * W + w]);
            out[(int64_t)(a - a0) * nl + b] = nd <= 4 ? orc_l2_element_abs(P, a, b) : 0.0;
        }
}

/* Class-4 condition rows [l0, l1) into out[(l - l0) * Dc + c]. */
void orc_class4_rows_abs(const orc_problem *P, int l0, int l1, double *out) {
    const int64_t Dc = orc_contracted_dim(P);
#pragma omp parallel for schedule(dynamic, 4)
    for (int l = l0; l < l1; ++l) orc_class4_row_abs(P, l, out + (int64_t)(l - l0) * Dc);
}

/* Full condition scale of a contracted continuum element: the sum of the
   magnitudes of every term of Eq. 8 followed by Eq. 7,
       sum_b |X(I^b)| sum_{m m'} |c_mn c_m'n' C^b_{m m'}|,
   the labels without a continuum index included term by term.  Rounding in
   any evaluation order of the contraction and the expansion (an FP64 one
   included) is bounded by a multiple of the unit roundoff of this scale. */
double orc_cc_element_cond(const orc_cc *c, int n, int j, int np, int jp) {
    const orc_problem *P = c->P;
    if (!c->with_abs) return NAN;
    const int ph = P->n_to, phk = P->n_to + 1, t = n * c->nsp + np;
    const int jg = P->n_to + j, jpg = P->n_to + jp;
    const orc_map *m = (j == jp) ? &c->same_abs : &c->diff_abs;
    double v = (j == jp) ? c->K0abs[t] : 0.0;
    for (int64_t i = 0; i < m->cap; ++i) {
        int s = m->slot[i];
        if (s < 0) continue;
        double x = (j == jp) ? orc_X(P, m->keys[i], ph, jg, -1, 0) : orc_X(P, m->keys[i], ph, jg, phk, jpg);
        v += m->blocks[(int64_t)s * m->bsz + t] * fabs(x);
    }
    return v;
}

/* The same for a whole group-pair block, written like orc_cc_expand. */
void orc_cc_expand_cond(const orc_cc *c, double *H, int64_t ld, int64_t row0, int64_t col0) {
    const orc_problem *P = c->P;
    const int cfg = P->g_cfirst[c->g], cng = P->g_ccount[c->g];
    const int cfp = P->g_cfirst[c->gp], cnp = P->g_ccount[c->gp];
#pragma omp parallel for schedule(dynamic, 1)
    for (int jj = 0; jj < cng; ++jj)
        for (int jjp = 0; jjp < cnp; ++jjp)
            for (int n = 0; n < c->ns; ++n)
                for (int np = 0; np < c->nsp; ++np) {
                    int64_t r = row0 + (int64_t)n * cng + jj, cl = col0 + (int64_t)np * cnp + jjp;
                    if (c->g == c->gp && r < cl) continue;
                    double v = orc_cc_element_cond(c, n, cfg + jj, np, cfp + jjp);
                    H[r * ld + cl] = v;
                    H[cl * ld + r] = v;
                }
}
