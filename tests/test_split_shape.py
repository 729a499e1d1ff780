"""The split expansion kernel's launch shape as the build plan chooses it
(host code of the library): tile width from a merged block's columns over
short K, 128 columns and 64-wide K stages from 32 K blocks (2048 labels) on,
so that every tile of a plan takes one K stage and a block's bits do not
depend on the columns it is merged with; forced widths and stages."""
import ctypes


def _shape():
    from paper_1709_03005_gb300 import build_ext
    lib = ctypes.CDLL(build_ext.build())
    fn = lib.hb_test_split_shape
    fn.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_int)] * 2
    fn.restype = ctypes.c_int

    def shape(n, kb, fc=0, fk=0):
        c, k = ctypes.c_int(), ctypes.c_int()
        rc = fn(n, kb, fc, fk, ctypes.byref(c), ctypes.byref(k))
        return rc, c.value, k.value
    return shape


def test_default_shapes():
    shape = _shape()
    # short K (the symmetry-blocked batch: 6 K blocks; the medium workload: 22)
    for kb in (1, 6, 22, 31):
        assert shape(1, kb) == (0, 32, 32)
        assert shape(32, kb) == (0, 32, 32)
        assert shape(33, kb) == (0, 64, 32)
        assert shape(64, kb) == (0, 64, 32)
        assert shape(65, kb) == (0, 128, 32)
        assert shape(1275, kb) == (0, 128, 32)
    # long K (the precision workload: 38 K blocks): one shape whatever the columns
    for kb in (32, 38, 116):
        for n in (1, 20, 64, 65, 1275):
            assert shape(n, kb) == (0, 128, 64)


def test_forced_shapes():
    shape = _shape()
    assert shape(20, 38, fc=32) == (0, 32, 32)          # narrow tiles always take 32-wide stages
    assert shape(20, 38, fc=64, fk=64) == (0, 64, 32)
    assert shape(20, 6, fc=128) == (0, 128, 32)
    assert shape(20, 6, fc=128, fk=64) == (0, 128, 64)
    assert shape(2000, 38, fk=32) == (0, 128, 32)
    assert shape(0, 6)[0] != 0 and shape(5, 0)[0] != 0
