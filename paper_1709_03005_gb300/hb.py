"""Python binding of the C ABI in include/hb.h (argument marshalling only).

Every function here forwards to libhb.so; there is no CPU fallback.  If the
library has not been built, `load()` raises.  Device memory for results comes
from PyTorch tensors; streams are PyTorch CUDA streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HB_OK, HB_ERR_INVALID_ARG, HB_ERR_CUDA, HB_ERR_OOM, HB_ERR_TIMEOUT, HB_ERR_NOT_CONVERGED, \
    HB_ERR_UNSUPPORTED = range(7)
HB_FP64, HB_MIXED = 0, 1
HB_PRECOND_DIAG, HB_PRECOND_MLP = 0, 1
HB_DIAG_TENSOR = 0x100
HB_NOALLOC_MAX_ROWS = 262144

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhb.so")


class hb_group(C.Structure):
    _fields_ = [("n_det", C.c_int32), ("n_state", C.c_int32), ("dets", C.c_void_p), ("ci", C.c_void_p),
                ("cont_first", C.c_int32), ("cont_count", C.c_int32), ("energy", C.c_void_p),
                ("n_csf", C.c_int32), ("csf_ptr", C.c_void_p), ("csf_det", C.c_void_p), ("csf_coef", C.c_void_p)]


class hb_problem(C.Structure):
    _fields_ = [("n_to", C.c_int32), ("n_co", C.c_int32), ("n_elec", C.c_int32), ("n_words", C.c_int32),
                ("cont_spin", C.c_int32), ("h", C.c_void_p), ("eri_tttt", C.c_void_p),
                ("eri_tttc", C.c_void_p), ("eri_ttcc", C.c_void_p), ("eri_tctc", C.c_void_p),
                ("n_groups", C.c_int32), ("groups", C.c_void_p), ("n_l2", C.c_int32),
                ("l2_dets", C.c_void_p), ("e_core", C.c_double), ("orb_irrep", C.c_void_p)]


class hb_options(C.Structure):
    _fields_ = [("split_slices", C.c_int32), ("validate", C.c_int32), ("autotune", C.c_int32),
                ("split_tile", C.c_int32), ("class4_states", C.c_int32), ("class4_threads", C.c_int32),
                ("class4_path", C.c_int32), ("mlp_stall_iters", C.c_int32), ("mlp_stall_log2", C.c_int32),
                ("diag_basis", C.c_int32), ("split_cols", C.c_int32),
                ("split_kstage", C.c_int32), ("reserved", C.c_int32 * 4)]


class hb_layout(C.Structure):
    _fields_ = [("dim", C.c_int64), ("contracted_dim", C.c_int64), ("n_l2", C.c_int64), ("l2_nnz", C.c_int64),
                ("tt_pairs", C.c_int64), ("tl2_pairs", C.c_int64), ("n_labels", C.c_int64),
                ("device_bytes", C.c_int64), ("n_groups", C.c_int32), ("n_words", C.c_int32),
                ("workspace_bytes", C.c_int64)]


class hb_blocks(C.Structure):
    _fields_ = [("Hcc", C.c_void_p), ("Hlc", C.c_void_p), ("l2_row_ptr", C.c_void_p), ("l2_col", C.c_void_p),
                ("l2_val", C.c_void_p)]


class hb_stats(C.Structure):
    _fields_ = [("ms_total", C.c_float), ("ms_target", C.c_float), ("ms_expand", C.c_float),
                ("ms_class4", C.c_float), ("ms_l2", C.c_float), ("ms_expand_gemm", C.c_float),
                ("expand_launches", C.c_int32), ("kernel_launches", C.c_int32), ("expand_flops", C.c_double),
                ("iterations", C.c_int32), ("mlp_fallbacks", C.c_int32), ("max_residual", C.c_double),
                ("ms_matvec", C.c_float), ("ms_rr", C.c_float), ("expand_tensor_flops", C.c_double),
                ("ms_gram", C.c_float), ("ms_combine", C.c_float), ("ms_class4_kernel", C.c_float),
                ("fp64_iterations", C.c_int32), ("mlp_loss", C.c_float), ("proj_gflop", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class hb_mlp_weights(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("width", C.c_int32), ("w1", C.c_void_p), ("b1", C.c_void_p),
                ("w2", C.c_void_p), ("b2", C.c_void_p), ("w3", C.c_void_p), ("b3", C.c_void_p)]


PAIR_DTYPE = np.dtype([("row", "<i4"), ("col", "<i4"), ("hole", "<i2", (2,)), ("part", "<i2", (2,)),
                       ("degree", "i1"), ("phase", "i1"), ("pad", "<i2", (3,))])
assert PAIR_DTYPE.itemsize == 24

EXPORTS = ["hb_init", "hb_init_shared", "hb_batch_create", "hb_batch_launch", "hb_batch_nodes",
           "hb_batch_destroy", "hb_query", "hb_group_offset", "hb_build_blocks", "hb_diag", "hb_classify",
           "hb_classify_noalloc", "hb_mlp_set", "hb_mlp_param_count", "hb_mlp_workspace_bytes", "hb_mlp_loss_grad",
           "hb_mlp_adam", "hb_mlp_train", "hb_mlp_train_params", "hb_mlp_predict", "hb_diag_features", "hb_batch_report", "hb_tuning_report",
           "hb_dump", "hb_target_diag", "hb_workspace_size", "hb_set_workspace",
           "hb_shard_coef_len", "hb_build_contract", "hb_build_expand",
           "hb_last_error", "hb_destroy"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libhb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1709_03005_gb300.build_ext.build()")
    lib = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    P = C.POINTER
    lib.hb_init.argtypes = [P(vp), P(hb_problem), P(hb_options), vp]
    lib.hb_query.argtypes = [vp, P(hb_layout)]
    lib.hb_group_offset.argtypes = [vp, i32]
    lib.hb_group_offset.restype = i64
    lib.hb_build_blocks.argtypes = [vp, i32, P(hb_blocks), P(hb_stats), vp]
    lib.hb_diag.argtypes = [vp, P(hb_blocks), i32, C.c_double, i32, i32, vp, vp, vp, P(hb_stats), vp]
    lib.hb_classify.argtypes = [vp, i32, vp, i32, i32, i32, i32, i32, i32, vp, vp, i64, P(i64), vp]
    lib.hb_mlp_set.argtypes = [vp, P(hb_mlp_weights)]
    lib.hb_last_error.argtypes = [vp]
    lib.hb_last_error.restype = C.c_char_p
    lib.hb_destroy.argtypes = [vp]
    lib.hb_destroy.restype = None
    for name in ["hb_init", "hb_query", "hb_build_blocks", "hb_diag", "hb_classify", "hb_mlp_set"]:
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class HBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hb error {code}: {msg}")
        self.code = code


def _check(rc, ctx=None):
    if rc != HB_OK:
        msg = load().hb_last_error(ctx)
        raise HBError(rc, msg.decode() if msg else "")


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr() if t is not None else 0)


# --------------------------------------------------------------------------
# the build
# --------------------------------------------------------------------------

def _marshal_problem(p, keep):
    """hb_problem (and its hb_group array) for a problem object; the numpy
    copies it points into are appended to `keep`."""
    def arr(x, dt):
        a = np.ascontiguousarray(x, dtype=dt)
        keep.append(a)
        return a

    gs = (hb_group * max(1, len(p.groups)))()
    for i, g in enumerate(p.groups):
        d = arr(g.dets, np.uint64)
        c = arr(g.ci, np.float64)
        en = getattr(g, "energy", None)
        e = arr(en, np.float64).ctypes.data if en is not None else None
        cp = getattr(g, "csf_ptr", None)
        if cp is not None:
            cp, cd, cc = arr(cp, np.int32), arr(g.csf_det, np.int32), arr(g.csf_coef, np.float64)
            csf = (cp.shape[0] - 1, cp.ctypes.data, cd.ctypes.data, cc.ctypes.data)
        else:
            csf = (0, None, None, None)
        gs[i] = hb_group(d.shape[0], c.shape[1], d.ctypes.data, c.ctypes.data, g.cont_first, g.cont_count, e, *csf)
    ptr = lambda a: a.ctypes.data
    l2 = arr(p.l2_dets, np.uint64) if p.l2_dets.shape[0] else None
    prob = hb_problem(p.n_to, p.n_co, p.n_elec, p.n_words, p.cont_spin,
                      ptr(arr(p.h, np.float64)), ptr(arr(p.eri_tttt, np.float64)),
                      ptr(arr(p.eri_tttc, np.float64)), ptr(arr(p.eri_ttcc, np.float64)),
                      ptr(arr(p.eri_tctc, np.float64)), len(p.groups), C.addressof(gs),
                      p.l2_dets.shape[0], ptr(l2) if l2 is not None else None, float(p.e_core),
                      ptr(arr(p.orb_irrep, np.int32)) if getattr(p, "orb_irrep", None) is not None else None)
    keep.append(gs)
    return prob, gs


def target_diag(problem, g, k, tol=1e-10, max_iter=400, stream=None):
    """hb_target_diag: the lowest k eigenpairs of the N-electron target
    Hamiltonian over group g's determinants.  Returns (energies [k],
    ci [n_det, k], stats), ready for the group's `energy` and `ci`
    (target-energy substitution)."""
    import torch
    lib = load()
    lib.hb_target_diag.argtypes = [C.POINTER(hb_problem), C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                   C.c_void_p, C.c_void_p, C.POINTER(hb_stats), C.c_void_p]
    lib.hb_target_diag.restype = C.c_int
    torch.cuda.init()
    keep = []
    prob, _ = _marshal_problem(problem, keep)
    nd = problem.groups[g].dets.shape[0] if 0 <= g < len(problem.groups) else 1   # the library checks g
    en = np.zeros(k)
    ci = np.zeros((nd, k))
    st = hb_stats()
    _check(lib.hb_target_diag(C.byref(prob), g, k, tol, max_iter, en.ctypes.data, ci.ctypes.data, C.byref(st),
                              _stream_handle(stream)))
    return en, ci, st


class Hamiltonian:
    """A staged problem (hb_init) whose blocks can be built and diagonalised.

    `problem` is any object with the fields of hb_problem (synth.Problem fits):
    n_to, n_co, n_elec, n_words, cont_spin, h, eri_*, groups (dets, ci,
    cont_first, cont_count), l2_dets, e_core.
    """

    def __init__(self, problem, split_slices=0, validate=True, stream=None, base=None, autotune=False,
                 split_tile=0, class4_states=0, class4_threads=0, class4_path=0, mlp_stall_iters=0,
                 mlp_stall_log2=0, diag_basis=0, split_cols=0, split_kstage=0):
        import torch
        self.lib = load()
        self.base = base        # keeps a borrowed-integral base context alive
        p = problem
        keep = []
        self._problem, gs = _marshal_problem(p, keep)
        opts = hb_options(split_slices, 1 if validate else 0, 1 if autotune else 0, split_tile, class4_states,
                          class4_threads, class4_path, mlp_stall_iters, mlp_stall_log2, diag_basis, split_cols,
                          split_kstage)
        self.ctx = C.c_void_p()
        torch.cuda.init()
        if base is None:
            rc = self.lib.hb_init(C.byref(self.ctx), C.byref(self._problem), C.byref(opts), _stream_handle(stream))
        else:
            self.lib.hb_init_shared.argtypes = [C.POINTER(C.c_void_p), C.POINTER(hb_problem), C.POINTER(hb_options),
                                                C.c_void_p, C.c_void_p]
            self.lib.hb_init_shared.restype = C.c_int
            rc = self.lib.hb_init_shared(C.byref(self.ctx), C.byref(self._problem), C.byref(opts), base.ctx,
                                         _stream_handle(stream))
        del keep, gs
        if rc != HB_OK:
            msg = self.lib.hb_last_error(None)
            raise HBError(rc, msg.decode() if msg else "")
        self.layout = hb_layout()
        _check(self.lib.hb_query(self.ctx, C.byref(self.layout)), self.ctx)
        self.group_offsets = [self.lib.hb_group_offset(self.ctx, g) for g in range(len(p.groups) + 1)]

    # sizes
    @property
    def dim(self):
        return self.layout.dim

    @property
    def contracted_dim(self):
        return self.layout.contracted_dim

    def allocate(self, device="cuda"):
        import torch
        L = self.layout
        Dc, nl = L.contracted_dim, L.n_l2
        return dict(
            Hcc=torch.zeros((Dc, Dc), dtype=torch.float64, device=device),
            Hlc=torch.zeros((nl, Dc), dtype=torch.float64, device=device),
            row_ptr=torch.zeros(nl + 1, dtype=torch.int64, device=device),
            col=torch.zeros(max(L.l2_nnz, 1), dtype=torch.int32, device=device),
            val=torch.zeros(max(L.l2_nnz, 1), dtype=torch.float64, device=device),
        )

    @staticmethod
    def blocks_struct(b):
        return hb_blocks(b["Hcc"].data_ptr(), b["Hlc"].data_ptr(), b["row_ptr"].data_ptr(),
                         b["col"].data_ptr(), b["val"].data_ptr())

    def build(self, precision=HB_FP64, blocks=None, stream=None, stats=True):
        b = blocks if blocks is not None else self.allocate()
        bs = self.blocks_struct(b)
        st = hb_stats()
        _check(self.lib.hb_build_blocks(self.ctx, precision, C.byref(bs), C.byref(st) if stats else None,
                                        _stream_handle(stream)), self.ctx)
        return b, st

    def diag(self, blocks, k, tol=1e-8, max_iter=200, precond=HB_PRECOND_DIAG, v0=None, evecs=None,
             stream=None, allow_not_converged=False):
        evals = np.zeros(k)
        bs = self.blocks_struct(blocks)
        st = hb_stats()
        rc = self.lib.hb_diag(self.ctx, C.byref(bs), k, tol, max_iter, precond, _ptr(v0),
                              evals.ctypes.data, _ptr(evecs), C.byref(st), _stream_handle(stream))
        if rc == HB_ERR_NOT_CONVERGED and allow_not_converged:
            return evals, st, False
        _check(rc, self.ctx)
        return evals, st, True

    def set_mlp(self, w1, b1, w2, b2, w3, b3):
        arrs = [np.ascontiguousarray(a, np.float32) for a in (w1, b1, w2, b2, w3, b3)]
        w = hb_mlp_weights(arrs[0].shape[1], arrs[0].shape[0], *[a.ctypes.data for a in arrs])
        _check(self.lib.hb_mlp_set(self.ctx, C.byref(w)), self.ctx)

    def set_mlp_params(self, packed):
        """Load a packed parameter vector (see unpack_mlp) for HB_PRECOND_MLP."""
        self.set_mlp(*unpack_mlp(packed))

    # sharded build (hb_build_contract / hb_build_expand)
    def shard_coef_len(self):
        self.lib.hb_shard_coef_len.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
        self.lib.hb_shard_coef_len.restype = C.c_int
        n = C.c_int64()
        _check(self.lib.hb_shard_coef_len(self.ctx, C.byref(n)), self.ctx)
        return n.value

    def build_contract(self, precision, rank, nranks, partial=None, stream=None):
        """This rank's contracted coefficient rows (a float64 device tensor)."""
        import torch
        self.lib.hb_build_contract.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                               C.POINTER(hb_stats), C.c_void_p]
        self.lib.hb_build_contract.restype = C.c_int
        if partial is None:
            partial = torch.empty(max(self.shard_coef_len(), 1), dtype=torch.float64, device="cuda")
        st = hb_stats()
        _check(self.lib.hb_build_contract(self.ctx, precision, rank, nranks, _ptr(partial), C.byref(st),
                                          _stream_handle(stream)), self.ctx)
        return partial, st

    def build_expand(self, precision, rank, nranks, reduced, blocks=None, stream=None):
        """This rank's share of the blocks from the reduced coefficient rows;
        blocks (zeros by default) keep what the rank does not write."""
        self.lib.hb_build_expand.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                             C.POINTER(hb_blocks), C.POINTER(hb_stats), C.c_void_p]
        self.lib.hb_build_expand.restype = C.c_int
        b = blocks if blocks is not None else self.allocate()
        bs = self.blocks_struct(b)
        st = hb_stats()
        _check(self.lib.hb_build_expand(self.ctx, precision, rank, nranks, _ptr(reduced), C.byref(bs), C.byref(st),
                                        _stream_handle(stream)), self.ctx)
        return b, st

    def workspace_size(self, precision=HB_MIXED, diag_k=0, precond=HB_PRECOND_DIAG, stream=None):
        """hb_workspace_size: device bytes the context's builds (and a solve
        for diag_k eigenpairs) take beyond hb_init."""
        self.lib.hb_workspace_size.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int64),
                                               C.c_void_p]
        self.lib.hb_workspace_size.restype = C.c_int
        out = C.c_int64()
        _check(self.lib.hb_workspace_size(self.ctx, precision, diag_k, precond, C.byref(out),
                                          _stream_handle(stream)), self.ctx)
        _check(self.lib.hb_query(self.ctx, C.byref(self.layout)), self.ctx)
        return out.value

    def set_workspace(self, buf):
        """hb_set_workspace with a caller-owned device tensor (kept alive here)."""
        self.lib.hb_set_workspace.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
        self.lib.hb_set_workspace.restype = C.c_int
        self._workspace = buf
        _check(self.lib.hb_set_workspace(self.ctx, C.c_void_p(buf.data_ptr()),
                                         buf.numel() * buf.element_size()), self.ctx)

    def dump(self, path):
        """hb_dump: a text description of the context into the file at path."""
        self.lib.hb_dump.argtypes = [C.c_void_p, C.c_char_p]
        self.lib.hb_dump.restype = C.c_int
        _check(self.lib.hb_dump(self.ctx, str(path).encode()), self.ctx)

    def tuning_report(self):
        """Launch shapes of this context's build plan (after a build), as text."""
        self.lib.hb_tuning_report.argtypes = [C.c_void_p, C.c_char_p, C.c_int32]
        self.lib.hb_tuning_report.restype = C.c_int32
        buf = C.create_string_buffer(4096)
        self.lib.hb_tuning_report(self.ctx, buf, len(buf))
        return buf.value.decode()

    def close(self):
        if getattr(self, "ctx", None) and self.ctx.value:
            self.lib.hb_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sharded_build(H, precision, rank, nranks, all_reduce, blocks=None, stream=None):
    """One rank's part of a sharded build (Section 3.1): the contraction over
    this rank's bra determinants, all_reduce(partial) summing the partial
    coefficient rows of every rank in place (torch.distributed.all_reduce over
    NCCL under torchrun), then this rank's tiles and L2 rows.  Returns the
    blocks: zero except where this rank wrote."""
    partial, _ = H.build_contract(precision, rank, nranks, stream=stream)
    all_reduce(partial)
    return H.build_expand(precision, rank, nranks, partial, blocks, stream=stream)[0]


def dense_from_blocks(b, dim=None):
    """Assemble the full symmetric matrix from the blocks (torch, on device)."""
    import torch
    Hcc, Hlc = b["Hcc"], b["Hlc"]
    Dc, nl = Hcc.shape[0], Hlc.shape[0]
    H = torch.zeros((Dc + nl, Dc + nl), dtype=torch.float64, device=Hcc.device)
    H[:Dc, :Dc] = Hcc
    H[Dc:, :Dc] = Hlc
    H[:Dc, Dc:] = Hlc.T
    if nl:
        rp = b["row_ptr"].to(torch.int64)
        counts = rp[1:] - rp[:-1]
        rows = torch.repeat_interleave(torch.arange(nl, device=Hcc.device), counts)
        nnz = int(rp[-1])
        H[Dc + rows, Dc + b["col"][:nnz].to(torch.int64)] = b["val"][:nnz]
    return H


# --------------------------------------------------------------------------
# excitation classification
# --------------------------------------------------------------------------

def classify(a, b, n_words, mode=0, cont_spin=0, max_degree=2, lower=False, cap=None, stream=None):
    """hb_classify on device uint64 tensors a [n_a, 2W], b [n_b, 2W].

    Returns (row_ptr [n_a+1] int64 tensor, records as a numpy structured array).
    """
    import torch
    lib = load()
    n_a, n_b = a.shape[0], b.shape[0]
    row_ptr = torch.zeros(n_a + 1, dtype=torch.int64, device=a.device)
    total = C.c_int64()
    rc = lib.hb_classify(_ptr(a), n_a, _ptr(b), n_b, n_words, mode, cont_spin, max_degree, 1 if lower else 0,
                         _ptr(row_ptr), None, 0, C.byref(total), _stream_handle(stream))
    if rc not in (HB_OK, HB_ERR_INVALID_ARG) or (rc == HB_ERR_INVALID_ARG and total.value == 0):
        _check(rc)
    n = total.value if cap is None else cap
    pairs = torch.zeros(max(n, 1) * PAIR_DTYPE.itemsize, dtype=torch.uint8, device=a.device)
    _check(lib.hb_classify(_ptr(a), n_a, _ptr(b), n_b, n_words, mode, cont_spin, max_degree, 1 if lower else 0,
                           _ptr(row_ptr), _ptr(pairs), n, C.byref(total), _stream_handle(stream)))
    torch.cuda.synchronize()
    rec = np.frombuffer(pairs.cpu().numpy().tobytes(), dtype=PAIR_DTYPE)[: total.value]
    return row_ptr, rec


def classify_noalloc(a, b, n_words, mode=0, cont_spin=0, max_degree=2, lower=False, pairs=None, stream=None):
    """hb_classify_noalloc on device uint64 tensors a [n_a, 2W], b [n_b, 2W].

    For callers that cannot allocate device memory: the row offsets live in the
    library's static device buffer (at most HB_NOALLOC_MAX_ROWS rows of a) and
    the caller provides the output buffer `pairs` (a uint8 device tensor of
    cap * 24 bytes).  Returns (number of pairs, records as a numpy array).
    """
    import torch
    lib = load()
    fn = lib.hb_classify_noalloc
    fn.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                   C.c_int32, C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p]
    fn.restype = C.c_int
    cap = pairs.numel() // PAIR_DTYPE.itemsize
    total = C.c_int64()
    _check(fn(_ptr(a), a.shape[0], _ptr(b), b.shape[0], n_words, mode, cont_spin, max_degree, 1 if lower else 0,
              _ptr(pairs), cap, C.byref(total), _stream_handle(stream)))
    torch.cuda.synchronize()
    rec = np.frombuffer(pairs.cpu().numpy().tobytes(), dtype=PAIR_DTYPE)[: total.value]
    return total.value, rec


# --------------------------------------------------------------------------
# learned preconditioner
# --------------------------------------------------------------------------

MLP_IN, MLP_WIDTH = 8, 64


def _mlp_fns():
    lib = load()
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    lib.hb_mlp_param_count.argtypes = [i32, i32]
    lib.hb_mlp_param_count.restype = C.c_int
    lib.hb_mlp_workspace_bytes.argtypes = [i64]
    lib.hb_mlp_workspace_bytes.restype = i64
    lib.hb_mlp_loss_grad.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp]
    lib.hb_mlp_loss_grad.restype = C.c_int
    lib.hb_mlp_adam.argtypes = [i64, vp, vp, vp, vp, i32, C.c_float, vp]
    lib.hb_mlp_adam.restype = C.c_int
    lib.hb_mlp_predict.argtypes = [vp, vp, i64, vp, vp]
    lib.hb_mlp_predict.restype = C.c_int
    lib.hb_mlp_train_params.argtypes = [vp, vp, vp, vp, i64, i64, i32, C.c_float, C.POINTER(C.c_float), vp]
    lib.hb_mlp_train_params.restype = C.c_int
    lib.hb_mlp_train.argtypes = [vp, C.POINTER(hb_mlp_dataset), vp, C.POINTER(hb_stats), vp]
    lib.hb_mlp_train.restype = C.c_int
    lib.hb_diag_features.argtypes = [vp, C.POINTER(hb_blocks), vp, i32, vp, vp]
    lib.hb_diag_features.restype = C.c_int
    return lib


def mlp_param_count():
    return _mlp_fns().hb_mlp_param_count(MLP_IN, MLP_WIDTH)


def mlp_loss_grad(params, feats, a, b, work=None, stream=None):
    """(loss, grads) of mean (w(f) a - b)^2 on the device (float32 tensors)."""
    import torch
    lib = _mlp_fns()
    n = feats.shape[0]
    if work is None:
        work = torch.empty(lib.hb_mlp_workspace_bytes(n), dtype=torch.uint8, device=feats.device)
    grads = torch.empty_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device=feats.device)
    _check(lib.hb_mlp_loss_grad(_ptr(params), _ptr(feats), _ptr(a), _ptr(b), n, _ptr(grads), _ptr(loss),
                                _ptr(work), _stream_handle(stream)))
    return loss, grads


def mlp_adam(params, grads, m, v, step, lr, stream=None):
    _check(_mlp_fns().hb_mlp_adam(params.numel(), _ptr(params), _ptr(grads), _ptr(m), _ptr(v), step, lr,
                                  _stream_handle(stream)))


class hb_mlp_dataset(C.Structure):
    _fields_ = [("n", C.c_int64), ("feats", C.c_void_p), ("a", C.c_void_p), ("b", C.c_void_p), ("batch", C.c_int64),
                ("steps", C.c_int32), ("lr", C.c_float)]


def mlp_train_ctx(H, params, feats, a, b, batch, steps, lr, stream=None):
    """hb_mlp_train: Adam on the data set with the context's memory; the trained
    network becomes H's preconditioner network.  Returns the stats (mlp_loss)."""
    d = hb_mlp_dataset(feats.shape[0], feats.data_ptr(), a.data_ptr(), b.data_ptr(), batch, steps, lr)
    st = hb_stats()
    _check(_mlp_fns().hb_mlp_train(H.ctx, C.byref(d), _ptr(params), C.byref(st), _stream_handle(stream)), H.ctx)
    return st


def mlp_train(params, feats, a, b, batch, steps, lr, stream=None):
    """hb_mlp_train_params: Adam over consecutive windows of the data set, params updated in place;
    returns the loss of the last window."""
    loss = C.c_float(0.0)
    _check(_mlp_fns().hb_mlp_train_params(_ptr(params), _ptr(feats), _ptr(a), _ptr(b), feats.shape[0], batch, steps, lr,
                                   C.byref(loss), _stream_handle(stream)))
    return loss.value


def mlp_predict(params, feats, stream=None):
    import torch
    out = torch.empty(feats.shape[0], dtype=torch.float32, device=feats.device)
    _check(_mlp_fns().hb_mlp_predict(_ptr(params), _ptr(feats), feats.shape[0], _ptr(out), _stream_handle(stream)))
    return out


def unpack_mlp(params):
    """Packed parameter vector -> (w1, b1, w2, b2, w3, b3) numpy arrays."""
    p = np.asarray(params, dtype=np.float32)
    W, I = MLP_WIDTH, MLP_IN
    o = 0
    out = []
    for shape in [(W, I), (W,), (W, W), (W,), (W,), (1,)]:
        sz = int(np.prod(shape))
        out.append(p[o:o + sz].reshape(shape))
        o += sz
    return out


def diag_features(H, blocks, theta, stream=None):
    """Features [q, dim, 8] (device float32) of every row for Ritz values theta."""
    import torch
    th = np.ascontiguousarray(theta, dtype=np.float64)
    out = torch.empty((len(th), H.dim, MLP_IN), dtype=torch.float32, device="cuda")
    bs = H.blocks_struct(blocks)
    _check(_mlp_fns().hb_diag_features(H.ctx, C.byref(bs), th.ctypes.data, len(th), _ptr(out),
                                       _stream_handle(stream)), H.ctx)
    return out



# --------------------------------------------------------------------------
# batched build (CUDA graph over many staged Hamiltonians)
# --------------------------------------------------------------------------

class Batch:
    """Stage several problems that share orbitals and integrals (the first one
    owns the staged integrals) and build them all with one graph launch."""

    def __init__(self, problems, precision=HB_MIXED, stream=None, **options):
        """options: hb_options fields for every context (split_tile, class4_path, ...)."""
        lib = load()
        lib.hb_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                        C.c_void_p]
        lib.hb_batch_create.restype = C.c_int
        lib.hb_batch_launch.argtypes = [C.c_void_p, C.POINTER(hb_stats), C.c_void_p]
        lib.hb_batch_launch.restype = C.c_int
        lib.hb_batch_nodes.argtypes = [C.c_void_p]
        lib.hb_batch_nodes.restype = C.c_int
        lib.hb_batch_destroy.argtypes = [C.c_void_p]
        lib.hb_batch_destroy.restype = None
        self.lib = lib
        self.hams = [Hamiltonian(problems[0], stream=stream, **options)]
        for p in problems[1:]:
            self.hams.append(Hamiltonian(p, validate=False, stream=stream, base=self.hams[0], **options))
        self.blocks = [h.allocate() for h in self.hams]
        n = len(self.hams)
        ctxs = (C.c_void_p * n)(*[h.ctx.value for h in self.hams])
        outs = (hb_blocks * n)(*[Hamiltonian.blocks_struct(b) for b in self.blocks])
        self._keep = (ctxs, outs)
        self.handle = C.c_void_p()
        _check(lib.hb_batch_create(C.byref(self.handle), ctxs, n, precision, outs, _stream_handle(stream)))
        self.positions = sum(h.dim * (h.dim + 1) / 2 for h in self.hams)

    @property
    def nodes(self):
        return self.lib.hb_batch_nodes(self.handle)

    def report(self):
        """The launch shapes the batch's autotuner chose, as text."""
        self.lib.hb_batch_report.argtypes = [C.c_void_p, C.c_char_p, C.c_int32]
        self.lib.hb_batch_report.restype = C.c_int32
        buf = C.create_string_buffer(4096)
        self.lib.hb_batch_report(self.handle, buf, len(buf))
        return buf.value.decode()

    def launch(self, stream=None, stats=True):
        st = hb_stats()
        _check(self.lib.hb_batch_launch(self.handle, C.byref(st) if stats else None, _stream_handle(stream)))
        return st

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.lib.hb_batch_destroy(self.handle)
            self.handle = C.c_void_p()
        for h in reversed(getattr(self, "hams", [])):
            h.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
