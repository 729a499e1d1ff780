"""Seeded synthetic scattering problems (inputs only).

This module builds the *inputs* of a close-coupling Hamiltonian build: orbital
integrals, target determinant lists with CI vectors, continuum-orbital ranges and
L2 determinant lists.  It holds none of the method's arithmetic (no Slater-Condon
rules, no contraction, no expansion): both the CPU oracle and the CUDA path read
what it produces.  The paper's own workloads (UKRMol H3PO4 and UKRMol+ BeH
integrals) are not available, so these seeded inputs stand in for them with the
shapes of the paper's problems: a CI-expanded target (Eq. 2) coupled to a set of
continuum orbitals, plus L2 configurations (Eq. 1).

Conventions shared by every consumer (they define the *input format*):

* spatial orbitals: target orbitals 0..n_to-1, continuum orbitals n_to..n_orb-1
  (continuum index j in 0..n_co-1 is global orbital n_to+j);
* a determinant is 2*W uint64 words: words 0..W-1 hold the alpha string, words
  W..2W-1 the beta string; bit p of a string is target orbital p;
* one-electron integrals h[p, q] over all n_orb orbitals (symmetric);
* two-electron integrals in chemists' notation (pq|rs), real, 8-fold symmetric,
  stored in four class arrays (at most two continuum indices ever occur in an
  (N+1)-electron function with a single continuum electron):
    eri_tttt[pair(p,q), pair(r,s)]          all four target
    eri_tttc[pair(p,q), r*n_co + j]         (pq|r j)
    eri_ttcc[pair(p,q), j*n_co + k]         (pq|j k), full square in (j, k)
    eri_tctc[r*n_co + j, s*n_co + k]        (r j|s k), full square
  where pair(p,q) = p(p+1)/2 + q for p >= q.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

ALPHA, BETA = 0, 1


def pair_index(p: int, q: int) -> int:
    if p < q:
        p, q = q, p
    return p * (p + 1) // 2 + q


@dataclass
class Group:
    """One target symmetry: determinants, CI vectors and its continuum range."""
    dets: np.ndarray        # (n_det, 2W) uint64
    ci: np.ndarray          # (n_det, n_state) float64, row-major c[m, n]
    cont_first: int         # first continuum orbital (0-based within continuum)
    cont_count: int         # number of continuum orbitals coupled to this group
    energy: np.ndarray | None = None   # target-state energies (target-energy substitution) or None
    # configuration state functions: CSF i = sum_k csf_coef[k] dets[csf_det[k]] for
    # csf_ptr[i] <= k < csf_ptr[i+1]; when given, ci is over the CSFs ([n_csf, n_state])
    csf_ptr: np.ndarray | None = None
    csf_det: np.ndarray | None = None
    csf_coef: np.ndarray | None = None
    spin: float | None = None           # total spin of the group's CSFs (information only)


@dataclass
class Problem:
    name: str
    n_to: int
    n_co: int
    n_elec: int             # N, electrons of the target
    n_words: int            # W, uint64 words per spin string
    cont_spin: int          # spin of the continuum electron (0 alpha, 1 beta)
    h: np.ndarray
    eri_tttt: np.ndarray
    eri_tttc: np.ndarray
    eri_ttcc: np.ndarray
    eri_tctc: np.ndarray
    groups: list
    l2_dets: np.ndarray     # (n_l2, 2W) uint64
    e_core: float = 0.0
    chol: np.ndarray | None = None   # packed-pair Cholesky factor (small problems)
    meta: dict = field(default_factory=dict)
    orb_irrep: np.ndarray | None = None   # spatial symmetry of every orbital (0..7, product XOR), or None

    @property
    def n_orb(self) -> int:
        return self.n_to + self.n_co

    @property
    def n_l2(self) -> int:
        return int(self.l2_dets.shape[0])

    @property
    def contracted_dim(self) -> int:
        return int(sum(g.ci.shape[1] * g.cont_count for g in self.groups))

    @property
    def dim(self) -> int:
        return self.contracted_dim + self.n_l2

    def full_eri(self) -> np.ndarray:
        """Full (pq|rs) tensor over all orbitals from the Cholesky factor (small only)."""
        assert self.chol is not None and self.n_orb <= 80
        n = self.n_orb
        P = np.zeros((n, n, self.chol.shape[1]))
        for p in range(n):
            for q in range(p + 1):
                P[p, q] = P[q, p] = self.chol[pair_index(p, q)]
        return np.einsum("pqk,rsk->pqrs", P, P)


# --------------------------------------------------------------------------
# determinant pools
# --------------------------------------------------------------------------

def occ_to_words(alpha_occ, beta_occ, W: int) -> np.ndarray:
    w = np.zeros(2 * W, dtype=np.uint64)
    for p in alpha_occ:
        w[p // 64] |= np.uint64(1) << np.uint64(p % 64)
    for p in beta_occ:
        w[W + p // 64] |= np.uint64(1) << np.uint64(p % 64)
    return w


def _excite(occ, n_orb, k):
    """All strings reached from `occ` by exactly k substitutions within 0..n_orb-1."""
    occ = tuple(occ)
    virt = tuple(sorted(set(range(n_orb)) - set(occ)))
    out = []
    for holes in itertools.combinations(occ, k):
        keep = [o for o in occ if o not in holes]
        for parts in itertools.combinations(virt, k):
            out.append(tuple(sorted(keep + list(parts))))
    return out


def sd_pool(n_alpha: int, n_beta: int, n_orb: int):
    """Reference (lowest orbitals filled) plus all singles and doubles, as (a, b)."""
    ra, rb = tuple(range(n_alpha)), tuple(range(n_beta))
    pool = [(ra, rb)]
    sa, sb = _excite(ra, n_orb, 1), _excite(rb, n_orb, 1)
    pool += [(a, rb) for a in sa] + [(ra, b) for b in sb]
    pool += [(a, rb) for a in _excite(ra, n_orb, 2)]
    pool += [(ra, b) for b in _excite(rb, n_orb, 2)]
    pool += [(a, b) for a in sa for b in sb]
    return pool


def sample_dets(rng, pool, n, W, include_reference=True):
    if n > len(pool):
        raise ValueError(f"asked for {n} determinants from a pool of {len(pool)}")
    if include_reference:
        idx = np.concatenate([[0], 1 + rng.choice(len(pool) - 1, n - 1, replace=False)])
    else:
        idx = rng.choice(len(pool), n, replace=False)
    return np.stack([occ_to_words(*pool[i], W) for i in idx]), idx


# --------------------------------------------------------------------------
# integrals
# --------------------------------------------------------------------------

def make_h(rng, n_to, n_co, cont_diag=(-3.0, -0.5), offdiag_sd=0.05, orb_irrep=None):
    n = n_to + n_co
    h = rng.normal(0.0, offdiag_sd, size=(n, n))
    h = np.tril(h, -1)
    h = h + h.T
    h[np.arange(n_to), np.arange(n_to)] = rng.uniform(-3.0, -0.5, size=n_to)
    h[np.arange(n_to, n), np.arange(n_to, n)] = rng.uniform(*cont_diag, size=n_co)
    if orb_irrep is not None:
        ir = np.asarray(orb_irrep)
        h[(ir[:, None] ^ ir[None, :]) != 0] = 0.0
    return h


def make_chol(rng, n_orb, rank, orb_irrep=None, return_irrep=False):
    """Packed-pair Cholesky-like factor L[pair(p,q), k] ~ N(0, 0.5/rank).  With
    orbital irreps every vector k carries an irrep and L[pair, k] vanishes
    unless the pair's irrep (XOR of its orbitals') is the vector's; with
    return_irrep the vectors' irreps are returned too."""
    npair = n_orb * (n_orb + 1) // 2
    L = rng.normal(0.0, np.sqrt(0.5 / rank), size=(npair, rank))
    if orb_irrep is not None:
        ir = np.asarray(orb_irrep)
        vec_irrep = rng.integers(0, 8, size=rank)
        vec_irrep[: max(1, rank // 8)] = 0   # keep totally symmetric vectors present
        pp, qq = np.tril_indices(n_orb)
        pi = np.empty(npair, dtype=np.int64)
        pi[_pair_index_array(pp, qq)] = ir[pp] ^ ir[qq]
        L[pi[:, None] != vec_irrep[None, :]] = 0.0
        if return_irrep:
            return L, vec_irrep
    return L


def _pair_index_array(p, q):
    """pair_index over arrays (p >= 0, q >= 0, either order)."""
    hi, lo = np.maximum(p, q), np.minimum(p, q)
    return hi * (hi + 1) // 2 + lo


def eri_classes(L, n_to, n_co, orb_irrep=None, vec_irrep=None):
    """The four class arrays of (pq|rs) = sum_k L[pq,k] L[rs,k].  With the
    orbitals' and the vectors' irreps (make_chol(..., return_irrep=True)) only
    the symmetry-allowed blocks are formed: rows and columns of pair irrep x
    against the vectors of irrep x, into arrays that are zero elsewhere."""
    Pt = n_to * (n_to + 1) // 2
    r_, j_ = np.meshgrid(np.arange(n_to), np.arange(n_co), indexing="ij")
    tc = _pair_index_array(n_to + j_.ravel(), r_.ravel())            # [r * n_co + j]
    j1, j2 = np.meshgrid(np.arange(n_co), np.arange(n_co), indexing="ij")
    cc = _pair_index_array(n_to + j1.ravel(), n_to + j2.ravel())     # [j * n_co + k]
    tt = np.arange(Pt)
    Ltt, Ltc = L[:Pt], L[tc]
    if orb_irrep is None:
        return Ltt @ Ltt.T, Ltt @ Ltc.T, Ltt @ L[cc].T, Ltc @ Ltc.T
    # orbitals sorted by irrep within the target and within the continuum: every
    # symmetry block of the class arrays is a contiguous sub-array
    ir = np.asarray(orb_irrep, dtype=np.int64)
    t_ir, c_ir = ir[:n_to], ir[n_to:]
    assert np.all(np.diff(t_ir) >= 0) and np.all(np.diff(c_ir) >= 0), "orbitals must be sorted by irrep"
    vec_irrep = np.asarray(vec_irrep)
    t_rng = {x: (int(np.searchsorted(t_ir, x)), int(np.searchsorted(t_ir, x, side="right"))) for x in range(8)}
    c_rng = {x: (int(np.searchsorted(c_ir, x)), int(np.searchsorted(c_ir, x, side="right"))) for x in range(8)}
    tt_ir = t_ir[np.tril_indices(n_to)[0]] ^ t_ir[np.tril_indices(n_to)[1]]
    tt_ir = tt_ir[np.argsort(_pair_index_array(*np.tril_indices(n_to)))]     # by packed pair index
    tttt = Ltt @ Ltt.T
    tttc = np.zeros((Pt, n_to, n_co))
    ttcc = np.zeros((Pt, n_co, n_co))
    tctc = np.zeros((n_to, n_co, n_to, n_co))
    Ltc3 = Ltc.reshape(n_to, n_co, -1)
    for x in range(8):
        k = np.flatnonzero(vec_irrep == x)
        rows = np.flatnonzero(tt_ir == x)
        if len(k) == 0:
            continue
        Lr = Ltt[rows][:, k]
        # (tt|tc): target orbital q of irrep u, continuum j of irrep u ^ x
        for u in range(8):
            (q0, q1), (a0, a1) = t_rng[u], c_rng[u ^ x]
            if q1 > q0 and a1 > a0 and len(rows):
                cols = Ltc3[q0:q1, a0:a1][:, :, k].reshape(-1, len(k))
                tttc[rows, q0:q1, a0:a1] = (Lr @ cols.T).reshape(len(rows), q1 - q0, a1 - a0)
        # (tt|cc): continuum j of irrep a, k of irrep a ^ x
        for a in range(8):
            (a0, a1), (b0, b1) = c_rng[a], c_rng[a ^ x]
            if a1 > a0 and b1 > b0 and len(rows):
                jj, kk = np.meshgrid(np.arange(a0, a1), np.arange(b0, b1), indexing="ij")
                cols = L[_pair_index_array(n_to + jj.ravel(), n_to + kk.ravel())][:, k]
                ttcc[rows, a0:a1, b0:b1] = (Lr @ cols.T).reshape(len(rows), a1 - a0, b1 - b0)
        # (tc|tc): (q of irrep t, j of irrep t ^ x) against (p of irrep u, j' of irrep u ^ x)
        blocks = [(t, *t_rng[t], *c_rng[t ^ x]) for t in range(8)]
        blocks = [b for b in blocks if b[2] > b[1] and b[4] > b[3]]
        for (t, q0, q1, a0, a1) in blocks:
            Lq = Ltc3[q0:q1, a0:a1][:, :, k].reshape(-1, len(k))
            for (u, p0, p1, b0, b1) in blocks:
                Lp = Ltc3[p0:p1, b0:b1][:, :, k].reshape(-1, len(k))
                tctc[q0:q1, a0:a1, p0:p1, b0:b1] = (Lq @ Lp.T).reshape(q1 - q0, a1 - a0, p1 - p0, b1 - b0)
    return (tttt, tttc.reshape(Pt, n_to * n_co), ttcc.reshape(Pt, n_co * n_co),
            tctc.reshape(n_to * n_co, n_to * n_co))


def orthonormal_ci(rng, n_det, n_state):
    g = rng.standard_normal((n_det, n_state))
    q, _ = np.linalg.qr(g)
    return np.ascontiguousarray(q)


# --------------------------------------------------------------------------
# problem families
# --------------------------------------------------------------------------

def make_problem(name, seed, n_to, n_co, n_elec, n_det, n_state, n_l2, rank,
                 cont_diag=(-3.0, -0.5), n_words=None, cont_spin=ALPHA,
                 n_groups=1, cont_ranges=None, keep_chol=None, e_core=0.0):
    """Single-spin-coupling problem: all groups share Ms and the continuum spin.

    cont_spin=ALPHA: targets have Ms=0 (N/2 alpha, N/2 beta), continuum alpha.
    cont_spin=BETA:  targets have Ms=+1 (N/2+1 alpha, N/2-1 beta), continuum beta.
    L2 determinants always carry N/2+1 alpha and N/2 beta electrons (Ms=+1/2).
    With several groups, target determinants are split disjointly among them.
    """
    rng = np.random.default_rng(seed)
    W = n_words or max(1, (n_to + 63) // 64)
    half = n_elec // 2
    if cont_spin == ALPHA:
        na, nb = half, n_elec - half
    else:
        na, nb = half + 1, n_elec - half - 1
    h = make_h(rng, n_to, n_co, cont_diag)
    L = make_chol(rng, n_to + n_co, rank)
    eri = eri_classes(L, n_to, n_co)

    pool = sd_pool(na, nb, n_to)
    total = n_det * n_groups
    dets, _ = sample_dets(rng, pool, total, W)
    groups = []
    for g in range(n_groups):
        d = dets[g * n_det:(g + 1) * n_det]
        ns = n_state[g] if isinstance(n_state, (list, tuple)) else n_state
        ci = orthonormal_ci(rng, n_det, ns)
        if cont_ranges is None:
            cf, cn = 0, n_co
        else:
            cf, cn = cont_ranges[g]
            if cf < 0 or cn < 1 or cf + cn > n_co:
                raise ValueError(f"continuum range {cf}+{cn} outside 0..{n_co}")
        groups.append(Group(np.ascontiguousarray(d), ci, cf, cn))

    l2pool = sd_pool(half + 1, n_elec - half, n_to)
    l2, _ = sample_dets(rng, l2pool, n_l2, W) if n_l2 > 0 else (np.zeros((0, 2 * W), np.uint64), None)
    keep = keep_chol if keep_chol is not None else (n_to + n_co) <= 40
    return Problem(name=name, n_to=n_to, n_co=n_co, n_elec=n_elec, n_words=W,
                   cont_spin=cont_spin, h=h, eri_tttt=eri[0], eri_tttc=eri[1],
                   eri_ttcc=eri[2], eri_tctc=eri[3], groups=groups,
                   l2_dets=np.ascontiguousarray(l2), e_core=float(e_core), chol=L if keep else None,
                   meta=dict(seed=seed, rank=rank))


# The five workloads.  Sizes follow the problem statement of each workload:
# C1 tiny FP64 build, C2 medium build + Davidson, C3 precision, C5 learned
# preconditioner (C3 family, more L2).  C4 (batched symmetry blocks) is built by
# make_batched_family below.
CONFIGS = {
    "c1": dict(name="c1_tiny", seed=1, n_to=10, n_co=20, n_elec=6, n_det=40, n_state=3,
               n_l2=50, rank=20),
    "c2": dict(name="c2_medium", seed=2, n_to=30, n_co=150, n_elec=10, n_det=2000,
               n_state=20, n_l2=5000, rank=60),
    "c3": dict(name="c3_precision", seed=3, n_to=40, n_co=400, n_elec=14, n_det=20000,
               n_state=50, n_l2=30000, rank=60, cont_diag=(0.0, 50.0)),
    "c5": dict(name="c5_learned", seed=5, n_to=40, n_co=400, n_elec=14, n_det=20000,
               n_state=50, n_l2=40000, rank=60, cont_diag=(0.0, 50.0)),
    # the L2-heavy shape of the paper's H3PO4 run (Section 4.1): contracted
    # dimension 712 (8 states x 89 continuum orbitals), 122103 L2 functions,
    # dimension 122815; the L2 x L2 block holds about 3.8e8 entries
    "h3po4": dict(name="l2_heavy_h3po4", seed=7, n_to=50, n_co=89, n_elec=14, n_det=2000, n_state=8,
                  n_l2=122103, rank=60),
    # a mid-size case that spans several GPU tiles with ragged tails and that the
    # oracle builds in full within seconds
    "mid": dict(name="mid_ragged", seed=11, n_to=12, n_co=37, n_elec=6, n_det=300,
                n_state=7, n_l2=700, rank=24),
}


def make_config(key: str, **overrides) -> Problem:
    kw = dict(CONFIGS[key])
    kw.update(overrides)
    return make_problem(**kw)


def make_tiny(seed, n_to=5, n_co=3, n_elec=4, n_det=6, n_state=2, n_l2=5, rank=6,
              n_groups=1, cont_spin=ALPHA, cont_ranges=None, n_words=None, e_core=0.0):
    """Tiny random problems for brute-force pinning (all integrals kept)."""
    return make_problem(f"tiny{seed}", seed, n_to, n_co, n_elec, n_det, n_state, n_l2,
                        rank, n_words=n_words, cont_spin=cont_spin, n_groups=n_groups,
                        cont_ranges=cont_ranges, keep_chol=True, e_core=e_core)


def random_det_pairs(rng, n_orb, n_alpha, n_beta, W, count, max_exc=3, orbitals=None):
    """Random determinant pairs (bra, ket) within `max_exc` substitutions.

    `orbitals`, if given, is the list of spatial orbitals the strings may use
    (e.g. orbitals straddling the 64-bit word boundaries).
    """
    orbs = np.arange(n_orb) if orbitals is None else np.asarray(orbitals)
    out = []
    for _ in range(count):
        a = rng.choice(orbs, n_alpha, replace=False)
        b = rng.choice(orbs, n_beta, replace=False)
        a2, b2 = set(a.tolist()), set(b.tolist())
        k = rng.integers(0, max_exc + 1)
        for _ in range(k):
            if rng.random() < 0.5 and len(set(orbs.tolist()) - a2) > 0:
                s = rng.choice(sorted(a2)); t = rng.choice(sorted(set(orbs.tolist()) - a2))
                a2.remove(s); a2.add(t)
            elif len(set(orbs.tolist()) - b2) > 0:
                s = rng.choice(sorted(b2)); t = rng.choice(sorted(set(orbs.tolist()) - b2))
                b2.remove(s); b2.add(t)
        out.append((occ_to_words(sorted(a.tolist()), sorted(b.tolist()), W),
                    occ_to_words(sorted(a2), sorted(b2), W)))
    bra = np.stack([o[0] for o in out])
    ket = np.stack([o[1] for o in out])
    return bra, ket


# --------------------------------------------------------------------------
# batched workload: 8 spatial symmetries x 2 spin couplings
# --------------------------------------------------------------------------

def _irrep_of(occ_a, occ_b, orb_irrep):
    x = 0
    for p in list(occ_a) + list(occ_b):
        x ^= int(orb_irrep[p])
    return x


def make_batched_family(seed=4, n_hams=16, n_to=40, cont_per_irrep=(50, 400), n_elec=8, rank=32,
                        dim_range=(500, 20000), max_det=600, max_states=16):
    """16 Hamiltonians of one D2h-like molecule: total symmetry Gamma in 0..7
    times two spin couplings (Ms = 0 targets + alpha continuum electron, and
    Ms = +1 targets + beta continuum electron).  Orbitals carry irreps (XOR is
    the group product); h and (pq|rs) vanish unless symmetry-allowed, so every
    Hamiltonian shares the same integrals.  Target group i holds determinants
    of irrep i and couples to the continuum orbitals of irrep i ^ Gamma (a
    contiguous range, orbitals ordered by irrep); two extra groups repeat an
    irrep with disjoint determinants (classes 5 and 6).  The target dimension of
    each Hamiltonian is log-uniform in dim_range: up to 60 % L2 (as far as the
    L2 pool of its symmetry allows), the rest contracted.  The groups enter in a
    fixed order, the two same-irrep pairs first, one state each while they fit;
    then states are added, up to max_states per group, until the contracted
    part reaches its share."""
    rng = np.random.default_rng(seed)
    n_irrep = 8
    t_irrep = np.repeat(np.arange(n_irrep), n_to // n_irrep)
    cont_counts = rng.integers(cont_per_irrep[0], cont_per_irrep[1] + 1, size=n_irrep)
    c_irrep = np.repeat(np.arange(n_irrep), cont_counts)
    cont_first = np.concatenate([[0], np.cumsum(cont_counts)[:-1]])
    n_co = int(cont_counts.sum())
    orb_irrep = np.concatenate([t_irrep, c_irrep])
    h = make_h(rng, n_to, n_co, orb_irrep=orb_irrep)
    L, vec_irrep = make_chol(rng, n_to + n_co, rank, orb_irrep=orb_irrep, return_irrep=True)
    eri = eri_classes(L, n_to, n_co, orb_irrep, vec_irrep)
    W = max(1, (n_to + 63) // 64)
    half = n_elec // 2
    pools = {}
    for spin in (ALPHA, BETA):
        na, nb = (half, half) if spin == ALPHA else (half + 1, half - 1)
        pool = sd_pool(na, nb, n_to)
        by_irrep = {i: [] for i in range(n_irrep)}
        for a, b in pool:
            by_irrep[_irrep_of(a, b, orb_irrep)].append((a, b))
        pools[spin] = by_irrep
    l2pool = sd_pool(half + 1, half, n_to)
    l2_by = {i: [] for i in range(n_irrep)}
    for a, b in l2pool:
        l2_by[_irrep_of(a, b, orb_irrep)].append((a, b))
    dims = np.exp(rng.uniform(np.log(dim_range[0]), np.log(dim_range[1]), size=n_hams)).astype(int)
    problems = []
    for hidx in range(n_hams):
        gam, spin = hidx % n_irrep, hidx // n_irrep
        target = int(dims[hidx])
        n_l2 = min(int(0.6 * target), len(l2_by[gam]))
        contracted = target - n_l2
        # groups: the same-irrep pairs of irreps 0 and 1, then the other irreps
        order = [0, 0, 1, 1] + list(range(2, n_irrep))
        width = [int(cont_counts[ir ^ gam]) for ir in order]
        take, cdim = 0, 0
        while take < len(order) and (take < 2 or cdim + width[take] <= contracted):
            cdim += width[take]
            take += 1
        irreps, width = order[:take], width[:take]
        ns = np.ones(take, dtype=int)
        grew = True
        while grew:
            grew = False
            for g in rng.permutation(take):
                if ns[g] < max_states and cdim + width[g] <= contracted + width[g] // 2:
                    ns[g] += 1
                    cdim += width[g]
                    grew = True
        used = {i: 0 for i in range(n_irrep)}
        groups = []
        for g, ir in enumerate(irreps):
            avail = pools[spin][ir]
            nd = min(max_det, max(int(ns[g]) + 2, len(avail) // 3))
            start = used[ir]
            if start + nd > len(avail):
                nd = len(avail) - start
            if nd < int(ns[g]) or nd <= 0:
                continue
            sel = avail[start:start + nd]
            used[ir] += nd
            perm = rng.permutation(len(sel))
            dets = np.stack([occ_to_words(*sel[i], W) for i in perm])
            ci = orthonormal_ci(rng, nd, int(min(ns[g], nd)))
            cir = ir ^ gam
            groups.append(Group(dets, ci, int(cont_first[cir]), int(cont_counts[cir])))
        l2sel = [l2_by[gam][i] for i in rng.choice(len(l2_by[gam]), n_l2, replace=False)] if n_l2 else []
        l2 = np.stack([occ_to_words(*x, W) for x in l2sel]) if l2sel else np.zeros((0, 2 * W), np.uint64)
        problems.append(Problem(name=f"batch_G{gam}_s{spin}", n_to=n_to, n_co=n_co, n_elec=n_elec, n_words=W,
                                cont_spin=spin, h=h, eri_tttt=eri[0], eri_tttc=eri[1], eri_ttcc=eri[2],
                                eri_tctc=eri[3], groups=groups, l2_dets=np.ascontiguousarray(l2),
                                meta=dict(seed=seed, gamma=gam, spin=spin, target_dim=target,
                                          orb_irrep=orb_irrep), orb_irrep=orb_irrep))
    return problems


# --------------------------------------------------------------------------
# spin-adapted target groups: configuration state functions (CSFs)
# --------------------------------------------------------------------------

def _fermion_apply(occ: tuple, ops):
    """Apply operators ((+1 create | -1 annihilate), spin orbital) right to
    left to the sorted spin-orbital tuple occ; returns (sign, tuple) or
    (0, None).  Input generation only (spin eigenfunctions)."""
    sign, cur = 1, list(occ)
    for kind, so in reversed(ops):
        i = 0
        while i < len(cur) and cur[i] < so:
            i += 1
        present = i < len(cur) and cur[i] == so
        if kind < 0:
            if not present:
                return 0, None
            del cur[i]
        else:
            if present:
                return 0, None
            cur.insert(i, so)
        sign *= -1 if i % 2 else 1
    return sign, tuple(cur)


def spin_eigenfunctions(alpha_occ_list, beta_occ_list, n_orb):
    """S^2 within the determinants of one spatial configuration (fixed Ms):
    returns (S values, eigenvectors as columns) with S from S(S+1).
    Determinants are alpha string then beta string in the canonical order of
    the input format (spin orbital s*n_orb + p, alpha first)."""
    dets = [tuple(sorted(list(a) + [n_orb + p for p in b])) for a, b in zip(alpha_occ_list, beta_occ_list)]
    index = {d: i for i, d in enumerate(dets)}
    n = len(dets)
    S2 = np.zeros((n, n))
    for j, d in enumerate(dets):
        na = sum(1 for so in d if so < n_orb)
        nb = len(d) - na
        sz = 0.5 * (na - nb)
        S2[j, j] += sz * sz + sz
        # S- S+ = sum_{p,q} a+_{q beta} a_{q alpha} a+_{p alpha} a_{p beta}
        for p in range(n_orb):
            for q in range(n_orb):
                sg, d2 = _fermion_apply(d, [(+1, n_orb + q), (-1, q), (+1, p), (-1, n_orb + p)])
                if sg and d2 in index:
                    S2[index[d2], j] += sg
    w, V = np.linalg.eigh(0.5 * (S2 + S2.T))
    S = 0.5 * (np.sqrt(np.maximum(4.0 * w + 1.0, 0.0)) - 1.0)
    return np.round(S * 2.0) / 2.0, V


def make_csf_problem(seed=12, n_to=8, n_co=6, n_elec=4, n_config=10, n_state=(2, 2), spins=(0.0, 1.0),
                     n_l2=12, rank=8, keep_chol=True):
    """Target groups given over configuration state functions: for each total
    spin S in `spins`, a group whose states are random orthonormal
    combinations of the CSFs of spin S built on the same sampled spatial
    configurations (singles and doubles of the closed-shell reference, all
    Ms = 0 determinants of each).  The groups share their determinant list
    and their continuum range: singlet and triplet targets coupled to the
    same continuum (classes 5 and 6 between target spins).  Each group carries
    csf_ptr, csf_det, csf_coef (CSF i = sum_k csf_coef[k] D[csf_det[k]] over
    csf_ptr[i] <= k < csf_ptr[i+1]) and ci over its CSFs."""
    rng = np.random.default_rng(seed)
    W = max(1, (n_to + 63) // 64)
    half = n_elec // 2
    h = make_h(rng, n_to, n_co)
    L = make_chol(rng, n_to + n_co, rank)
    eri = eri_classes(L, n_to, n_co)
    pool = sd_pool(half, n_elec - half, n_to)
    configs = {}
    for a, b in pool:
        docc = tuple(sorted(set(a) & set(b)))
        socc = tuple(sorted(set(a) ^ set(b)))
        configs.setdefault((docc, socc), None)
    keys = list(configs)
    pick = [0] + list(1 + rng.choice(len(keys) - 1, min(n_config, len(keys)) - 1, replace=False))
    dets, csfs = [], {S: [] for S in spins}
    for ci_ in pick:
        docc, socc = keys[ci_]
        k = len(socc)
        n_open_a = (k + (half - (n_elec - half))) // 2
        alist, blist = [], []
        for up in itertools.combinations(socc, n_open_a):
            a = tuple(sorted(docc + up))
            b = tuple(sorted(docc + tuple(o for o in socc if o not in up)))
            alist.append(a)
            blist.append(b)
        base = len(dets)
        for a, b in zip(alist, blist):
            dets.append(occ_to_words(a, b, W))
        Svals, V = spin_eigenfunctions(alist, blist, n_to)
        for c in range(V.shape[1]):
            if Svals[c] in csfs:
                idx = [base + i for i in range(len(alist)) if abs(V[i, c]) > 1e-12]
                csfs[Svals[c]].append((idx, [V[i - base, c] for i in idx]))
    dets = np.stack(dets)
    groups = []
    for g, S in enumerate(spins):
        lst = csfs[S]
        ns = n_state[g] if isinstance(n_state, (list, tuple)) else n_state
        if len(lst) < ns:
            raise ValueError(f"only {len(lst)} CSFs of spin {S}")
        ptr = np.zeros(len(lst) + 1, np.int32)
        for i, (idx, _) in enumerate(lst):
            ptr[i + 1] = ptr[i] + len(idx)
        cdet = np.concatenate([np.asarray(i, np.int32) for i, _ in lst])
        coef = np.concatenate([np.asarray(c, np.float64) for _, c in lst])
        groups.append(Group(dets.copy(), orthonormal_ci(rng, len(lst), ns), 0, n_co, csf_ptr=ptr, csf_det=cdet,
                            csf_coef=coef, spin=S))
    l2pool = sd_pool(half + 1, n_elec - half, n_to)
    l2, _ = sample_dets(rng, l2pool, n_l2, W) if n_l2 > 0 else (np.zeros((0, 2 * W), np.uint64), None)
    return Problem(name=f"csf{seed}", n_to=n_to, n_co=n_co, n_elec=n_elec, n_words=W, cont_spin=ALPHA, h=h,
                   eri_tttt=eri[0], eri_tttc=eri[1], eri_ttcc=eri[2], eri_tctc=eri[3], groups=groups,
                   l2_dets=np.ascontiguousarray(l2), chol=L if keep_chol else None,
                   meta=dict(seed=seed, rank=rank, spins=list(spins)))
