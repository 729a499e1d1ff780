"""Helpers shared by the GPU parity tests (build through the C ABI, compare with
the oracle).

Element criterion (per element):

    |G - R| <= rel * max(|R|, 1e-6 * max|R_block|)          (floored relative)
 or |G - R| <= fallback * cond                               (cancellation)

where cond is the oracle's full condition scale of that element: the sum of
the magnitudes of every term its value adds up (for a continuum element every
term of the contraction, Eq. 8, and of the expansion, Eq. 7; for class 4 every
term of Eq. 5; for L2 every Slater-Condon term).  The second clause is looser
than the first only for elements whose value cancels below (fallback / rel) *
cond; `check_elements` counts those.  The constants are error bounds of the
arithmetic, checked against the measured worst cases:

  FP64 (rel 1e-12): fallback 64 u (u = 2^-53), the rounding of two summation
    orders of the same terms (measured worst 56 u at dimension 50000); it
    covers elements with |R| < 7.1e-3 cond.
  mixed continuum (rel 1e-10): fallback 3e-11, the split products' operands
    are exact to 2^-42 of the scale of their row of labels (measured worst
    1.5e-11); it covers elements with |R| < 0.3 cond.
  mixed class 4 (double-float or split-bf16 tensor cores, rel 1e-10):
    fallback 3e-12 (measured worst 1.6e-12); and, on the tensor cores, whose
    operands are quantised against the largest integral of each continuum
    orbital and the largest coefficient of each state, |G - R| <= 1e-12
    max|R_block| for elements far below those scales (measured worst 2.4e-13,
    2^-42, of the block scale).
  The L2 block is FP64 on both paths (rel 1e-12, fallback 64 u).
Structural zeros (oracle value exactly 0) must be exact zeros in every block.
"""
import numpy as np

from oracle import coracle

U = np.finfo(np.float64).eps / 2
FP64_FALLBACK = 64 * U
MIXED_CC_FALLBACK = 3e-11
MIXED_C4_FALLBACK = 3e-12
MIXED_C4_TC_ABS = 1e-12


def gpu_dense(problem, precision=0, **kw):
    import torch
    from paper_1709_03005_gb300 import hb
    H = hb.Hamiltonian(problem, **kw)
    blocks, st = H.build(precision)
    torch.cuda.synchronize()
    D = hb.dense_from_blocks(blocks).cpu().numpy()
    H.close()
    return D, st, blocks


def block_slices(o: coracle.Oracle):
    """(name, row slice, col slice) of the class blocks of the dense matrix."""
    Dc, dim = o.Dc, o.dim
    out = [("cc", slice(0, Dc), slice(0, Dc)), ("l2c", slice(Dc, dim), slice(0, Dc)),
           ("l2", slice(Dc, dim), slice(Dc, dim))]
    return [b for b in out if b[1].stop > b[1].start and b[2].stop > b[2].start]


def check_elements(g, r, cond, rel, fallback, what, blockmax=None, zeros=True, abs_frac=None):
    """Assert the element criterion above (with abs_frac: also accept
    |G - R| <= abs_frac * max|R_block|); returns (fraction within rel of |R|,
    fraction within the floored bound, number of elements passing only by the
    other clauses, worst |G - R| / cond)."""
    g, r, cond = np.asarray(g), np.asarray(r), np.asarray(cond)
    if r.size == 0:
        return 1.0, 1.0, 0, 0.0
    bm = np.abs(r).max() if blockmax is None else blockmax
    d = np.abs(g - r)
    floored = d <= rel * np.maximum(np.abs(r), 1e-6 * bm)
    canc = d <= fallback * cond
    if abs_frac is not None:
        canc |= d <= abs_frac * bm
    bad = ~(floored | canc)
    worst = float((d / np.maximum(cond, 1e-300)).max())
    assert not bad.any(), (f"{what}: {bad.sum()} of {d.size} elements off (max |d| {d.max():.3e}, "
                           f"worst |d|/cond {worst:.3e}, block scale {bm:.3e})")
    if zeros:
        z = r == 0.0
        assert np.all(g[z] == 0.0), f"{what}: {int((g[z] != 0).sum())} structural zeros are not exact zeros"
    strict = float((d <= rel * np.abs(r)).mean())
    return strict, float(floored.mean()), int((~floored).sum()), worst


def assert_blocks_close(G, R, o, rel=1e-12, what="", S=None, mixed=False):
    """Every block of the dense GPU matrix G against the oracle's R with the
    element criterion; S (the oracle's condition scales) is computed if not
    given.  FP64 by default; mixed=True uses the mixed path's constants (its L2
    block is FP64)."""
    S = o.condition() if S is None else S
    fb = {"cc": MIXED_CC_FALLBACK, "l2c": MIXED_C4_FALLBACK} if mixed else {"cc": FP64_FALLBACK, "l2c": FP64_FALLBACK}
    fb["l2"] = FP64_FALLBACK
    rl = {"cc": rel, "l2c": rel, "l2": 1e-12}
    out = {}
    for name, rs, cs in block_slices(o):
        out[name] = check_elements(G[rs, cs], R[rs, cs], S[rs, cs], rl[name], fb[name], f"{what} block {name}",
                                   abs_frac=MIXED_C4_TC_ABS if mixed and name == "l2c" else None)
    return out


def l2_csr_cond(o, rp, cols, chunk=512):
    """The oracle's condition scales at the positions of an L2 CSR pattern."""
    n = len(rp) - 1
    out = np.empty(int(rp[-1]))
    for a0 in range(0, n, chunk):
        a1 = min(n, a0 + chunk)
        S = o.l2_rows_abs(a0, a1)
        for a in range(a0, a1):
            out[rp[a]:rp[a + 1]] = S[a - a0, cols[rp[a]:rp[a + 1]]]
    return out


def sampled_checks(P, o, cc, b, rng, precision, n_cc=400, n_rows=12, what=""):
    """Sampled continuum elements, whole class-4 rows and whole L2 rows of the
    built blocks b against the oracle.  Returns the fraction of sampled
    continuum elements within 1e-10 of their own magnitude."""
    mixed = precision == 1
    rel = 1e-10 if mixed else 1e-12
    ns, nco = P.groups[0].ci.shape[1], P.n_co
    idx = [(int(n), int(j), int(n_), int(j if rng.random() < 0.1 else jp))
           for n, n_, j, jp in zip(*[rng.integers(0, m, n_cc) for m in (ns, ns, nco, nco)])]
    ref = np.array([cc.element(*t) for t in idx])
    cond = np.array([cc.element_cond(*t) for t in idx])
    Hcc = b["Hcc"]
    got = np.array([float(Hcc[n * nco + j, n_ * nco + jp]) for n, j, n_, jp in idx])
    bm = float(Hcc.abs().max())
    _, _, n_canc, worst = check_elements(got, ref, cond, rel, MIXED_CC_FALLBACK if mixed else FP64_FALLBACK,
                                         f"{what} cc sampled", blockmax=bm)
    strict10 = float(np.mean(np.abs(got - ref) <= 1e-10 * np.abs(ref)))
    # The mixed error stays below 3e-11 of the element's condition scale
    # (the fallback clause; measured at most 2.0e-11, on the L2-heavy
    # workload), so an element whose terms cancel by at most a factor of 3
    # meets the relative bound itself: every such element is held to it.
    d = np.abs(got - ref)
    ratio = cond / np.maximum(np.abs(ref), 1e-300)
    plain = ratio <= 3.0
    off = plain & (d > rel * np.abs(ref))
    assert not off.any(), (f"{what}: {int(off.sum())} of {int(plain.sum())} continuum elements with condition scale "
                           f"within 3 of their magnitude beyond {rel:g} relative")
    stats = []
    for lim in (3, 10, 100):
        sel = ratio <= lim
        if sel.any():
            stats.append(f"cond <= {lim}|ref|: {int(sel.sum())}, max rel {float((d[sel] / np.abs(ref[sel])).max()):.1e}")
    print(f"{what}: {100 * strict10:.2f} % of sampled continuum elements within 1e-10 of their magnitude; "
          f"{n_canc} by the cancellation clause; |d|/cond max {worst:.1e}, median "
          f"{float(np.median(d / np.maximum(cond, 1e-300))):.1e}; cond/|ref| median {float(np.median(ratio)):.0f}; "
          + "; ".join(stats))
    rows = np.sort(rng.choice(P.n_l2, n_rows, replace=False))
    ref4 = np.stack([o.class4_row(int(l)) for l in rows])
    cond4 = np.stack([o.class4_rows_abs(int(l), int(l) + 1)[0] for l in rows])
    g4 = b["Hlc"][rows].cpu().numpy()
    check_elements(g4, ref4, cond4, rel, MIXED_C4_FALLBACK if mixed else FP64_FALLBACK, f"{what} class 4 rows",
                   blockmax=float(b["Hlc"].abs().max()), abs_frac=MIXED_C4_TC_ABS if mixed else None)
    rp = b["row_ptr"].cpu().numpy()
    for a in rng.choice(P.n_l2, n_rows, replace=False):
        row = o.l2_rows(int(a), int(a) + 1)[0]
        rcond = o.l2_rows_abs(int(a), int(a) + 1)[0]
        cols = b["col"][rp[a]:rp[a + 1]].cpu().numpy()
        vals = b["val"][rp[a]:rp[a + 1]].cpu().numpy()
        dense = np.zeros(P.n_l2)
        dense[cols] = vals
        check_elements(dense, row, rcond, 1e-12, FP64_FALLBACK, f"{what} L2 row {a}")
        assert set(cols.tolist()) >= set(np.nonzero(row)[0].tolist())
    return strict10
