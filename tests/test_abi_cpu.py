"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function include/chessfad.h declares, and rejects bad
arguments with the documented status codes before launching anything."""
import ctypes
import os
import re

import pytest

import paper_2410_22575_gb300 as cf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"CHESSFAD_API\s+[\w\s\*]*?\b(chessfad_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = cf.load()
    names = _declared()
    assert len(names) >= 10
    for name in sorted(names):
        assert hasattr(lib, name), name


def test_version_and_strerror():
    assert cf.chessfad_version() >= 100
    assert cf.strerror(0) == "success"
    for code in range(-12, 0):
        assert cf.strerror(code) != "unknown status"
    assert cf.strerror(-99) == "unknown status"


def test_argument_errors_without_gpu():
    lib = cf.load()
    dummy = ctypes.c_void_p(16)
    # function id, size, batch, chunk, precision, null pointers: rejected on the host
    assert lib.chessfad_hvp(3, 8, 4, 4, dummy, dummy, dummy, None, 0, None) == -1
    assert lib.chessfad_hvp(0, 0, 4, 4, dummy, dummy, dummy, None, 0, None) == -2
    assert lib.chessfad_hvp(0, 513, 4, 4, dummy, dummy, dummy, None, 0, None) == -2
    assert lib.chessfad_hvp(0, 8, -1, 4, dummy, dummy, dummy, None, 0, None) == -3
    assert lib.chessfad_hvp(0, 8, 4, 3, dummy, dummy, dummy, None, 0, None) == -4
    assert lib.chessfad_hvp(0, 8, 4, 64, dummy, dummy, dummy, None, 0, None) == -4
    assert lib.chessfad_hvp(0, 8, 4, 4, None, dummy, dummy, None, 0, None) == -5
    assert lib.chessfad_hvp(0, 8, 4, 4, dummy, None, dummy, None, 0, None) == -5
    assert lib.chessfad_hessian(0, 8, 4, 4, dummy, None, None, 0, None) == -5
    assert lib.chessfad_hvp(0, 8, 4, 4, dummy, dummy, dummy, None, 7, None) == -7
    # Fletcher-Powell needs parameters with ld >= n
    assert lib.chessfad_hvp(2, 8, 4, 4, dummy, dummy, dummy, None, 0, None) == -6
    p = cf.FPParams(16, 16, 16, 4)
    assert lib.chessfad_hvp(2, 8, 4, 4, dummy, dummy, dummy, ctypes.byref(p), 0, None) == -6
    # batch == 0 is a no-op that succeeds without touching the device
    assert lib.chessfad_hvp(0, 8, 0, 4, None, None, None, None, 0, None) == 0
    # bad launch configurations
    bad = cf.Config(4, 3, 256)
    assert lib.chessfad_hvp_config(0, 8, 4, ctypes.byref(bad), dummy, dummy, dummy, None, 0, None) == -9
    bad = cf.Config(4, 4, 1024)
    assert lib.chessfad_hvp_config(0, 8, 4, ctypes.byref(bad), dummy, dummy, dummy, None, 0, None) == -9
    bad = cf.Config(5, 4, 256)
    assert lib.chessfad_hvp_config(0, 8, 4, ctypes.byref(bad), dummy, dummy, dummy, None, 0, None) == -4
    bad = cf.Config(4, 0, 0, 4, 0)  # unknown method
    assert lib.chessfad_hvp_config(0, 8, 4, ctypes.byref(bad), dummy, dummy, dummy, None, 0, None) == -9
    bad = cf.Config(32, 0, 0, cf.POINT, 0)  # one-thread-per-point kernels: chunk sizes 1..16
    assert lib.chessfad_hvp_config(0, 8, 4, ctypes.byref(bad), dummy, dummy, dummy, None, 0, None) == -4
    for c in (1, 2, 32):  # seed-sparse kernels: chunk sizes 4, 8 and 16 only
        bad = cf.Config(c, 0, 0, cf.SYMMETRIC_SPARSE, 32)
        assert lib.chessfad_hvp_config(0, 8, 4, ctypes.byref(bad), dummy, dummy, dummy, None, 0, None) == -4
    for tpp in (4, 48, 512):
        bad = cf.Config(4, 0, 0, cf.SYMMETRIC, tpp)
        assert lib.chessfad_hvp_config(0, 8, 4, ctypes.byref(bad), dummy, dummy, dummy, None, 0, None) == -9


def test_host_pipeline_argument_errors_without_gpu():
    lib = cf.load()
    d = ctypes.c_void_p(16)
    args = [d] * 6
    assert lib.chessfad_hvp_host(3, 8, 4, 4, *args, None, 0, 0, None) == -1
    assert lib.chessfad_hvp_host(0, 8, -1, 4, *args, None, 0, 0, None) == -3
    assert lib.chessfad_hvp_host(0, 8, 4, 3, *args, None, 0, 0, None) == -4
    assert lib.chessfad_hvp_host(0, 8, 4, 4, *args, None, 0, 65, None) == -9
    assert lib.chessfad_hvp_host(0, 8, 4, 4, *args, None, 0, -1, None) == -9
    assert lib.chessfad_hvp_host(0, 8, 4, 4, None, d, d, d, d, d, None, 0, 0, None) == -5
    assert lib.chessfad_hvp_host(0, 8, 4, 4, d, d, d, d, d, None, None, 0, 0, None) == -5
    assert lib.chessfad_hvp_host(2, 8, 4, 4, *args, None, 0, 0, None) == -6
    assert lib.chessfad_hvp_host(0, 8, 0, 4, None, None, None, None, None, None, None, 0, 0, None) == 0


def test_batch_beyond_one_launch_grid_is_rejected_without_gpu():
    # a launch grid holds at most 2^31 - 1 blocks; a batch needing more is
    # rejected on the host (never truncated to 32 bits), for every method
    lib = cf.load()
    d = ctypes.c_void_p(16)
    big = 1 << 40
    for n, cfg in ((512, cf.Config(16, 32, 256, cf.PLAIN, 0)), (512, cf.Config(8, 0, 0, cf.SYMMETRIC, 8)),
                   (16, cf.Config(4, 0, 256, cf.POINT, 0))):
        assert lib.chessfad_hvp_config(0, n, big, ctypes.byref(cfg), d, d, d, None, 0, None) == -3, cfg.as_dict()
    one = cf.Config(1, 1, 256, cf.PLAIN, 0)  # n = 1 in compensated FP32 (the FP64-evaluated path)
    assert lib.chessfad_hvp_config(0, 1, 1 << 45, ctypes.byref(one), d, d, d, None, 1, None) == -3


def test_compensated_primitives_argument_errors_without_gpu():
    # every rejection happens on the host, before a launch (no device pointer
    # is ever dereferenced: the calls below launch nothing)
    lib = cf.load()
    d = ctypes.c_void_p(16)
    assert lib.chessfad_eft(d, d, -1, d, d, d, d, None) == -3
    assert lib.chessfad_eft(None, d, 8, d, d, d, d, None) == -5
    assert lib.chessfad_eft(d, None, 8, d, d, d, d, None) == -5
    assert lib.chessfad_eft(None, None, 0, None, None, None, None, None) == 0
    assert lib.chessfad_compensated_rows(d, d, -1, 8, 4, 1, d, None) == -3
    assert lib.chessfad_compensated_rows(d, d, 4, -1, 4, 1, d, None) == -3
    assert lib.chessfad_compensated_rows(d, d, 2**62, 8, 4, 1, d, None) == -3
    for lanes in (0, 3, 6, 64):
        assert lib.chessfad_compensated_rows(d, d, 4, 8, lanes, 1, d, None) == -9
    assert lib.chessfad_compensated_rows(d, d, 4, 8, 4, 0, d, None) == -9
    assert lib.chessfad_compensated_rows(d, d, 4, 8, 4, 1, None, None) == -5
    assert lib.chessfad_compensated_rows(None, d, 4, 8, 4, 1, d, None) == -5
    assert lib.chessfad_compensated_rows(None, None, 0, 8, 4, 1, None, None) == 0


def test_untuned_default_is_symmetric_at_the_sec5_chunk():
    """Untuned default: the symmetric method for n >= 4 with csize near the
    Sec. V optimum sqrt(n/2) (a power of two at or above it, capped by the
    precision's register budget); the plain method below n = 4."""
    import math

    for fn in (0, 1, 2):
        for prec in (0, 1):
            for n in (4, 8, 16, 32, 64, 128, 256, 512):
                c = cf.chessfad_default_config(fn, n, 4096, prec)
                assert c.method == cf.SYMMETRIC, (fn, prec, n)
                target = math.sqrt(n / 2)
                assert c.csize >= min(target, 4) and (c.csize == 1 or c.csize / 2 < target), (n, c.csize)
            for n in (1, 2, 3):
                assert cf.chessfad_default_config(fn, n, 4096, prec).method == cf.PLAIN


def test_default_threads_per_point_capped_by_items():
    """The untuned symmetric default never gives a point more threads than it
    has (row, chunk) items C nch (nch+1)/2 (rounded up to a power of two, at
    least 8): at n = 4, c = 2 a point has 6 items, so 8 threads."""
    for fn in (0, 1, 2):
        for prec in (0, 1):
            for n in (4, 5, 8, 12, 16, 64, 256):
                for batch in (1, 100, 4096, 1 << 20):
                    c = cf.chessfad_default_config(fn, n, batch, prec)
                    nch = -(-n // c.csize)
                    items = c.csize * nch * (nch + 1) // 2
                    cap = max(8, 1 << (items - 1).bit_length())
                    assert 8 <= c.threads_per_point <= min(256, cap), (fn, prec, n, batch, c.as_dict())
    assert cf.chessfad_default_config(0, 4, 4096, 0).threads_per_point == 8


def test_csize0_chunk_follows_the_method():
    """csize 0 with an explicit method: the symmetric methods take the Sec. V
    chunk sqrt(n/2), the one-thread-per-point method the plain method's
    register-resident chunk; method 0 means the default method."""
    import math

    for fn in (0, 1, 2):
        for prec in (0, 1):
            d = cf.chessfad_default_config(fn, 64, 4096, prec)
            assert cf.chessfad_resolve_config(fn, 64, 4096, prec, cf.Config(0, 0, 0, 0, 0)).as_dict() == d.as_dict()
            assert cf.chessfad_resolve_config(fn, 64, 4096, prec).as_dict() == d.as_dict()
            cap = 4 if (fn == 2 and prec == 0) else (8 if prec == 0 else 16)  # register budget
            s = cf.chessfad_resolve_config(fn, 64, 4096, prec, cf.Config(0, 0, 0, cf.SYMMETRIC, 0))
            assert s.method == cf.SYMMETRIC and s.csize == min(cap, 8) and 8 >= math.sqrt(32) > 4
            p = cf.chessfad_resolve_config(fn, 64, 4096, prec, cf.Config(0, 0, 0, cf.POINT, 0))
            assert p.method == cf.POINT and p.csize == cap
            sp = cf.chessfad_resolve_config(fn, 64, 4096, prec, cf.Config(0, 0, 0, cf.SYMMETRIC_SPARSE, 0))
            assert sp.method == cf.SYMMETRIC_SPARSE and sp.csize in (4, 8, 16)
            # an explicit chunk size with method 0 is the plain method
            assert cf.chessfad_resolve_config(fn, 64, 4096, prec, cf.Config(4, 1, 256, 0, 0)).method == cf.PLAIN
    with pytest.raises(cf.ChessfadError):
        cf.chessfad_resolve_config(0, 64, 4096, 0, cf.Config(3, 0, 0, 0, 0))


@pytest.mark.parametrize("fn", [0, 1, 2])
@pytest.mark.parametrize("prec", [0, 1])
def test_default_config_host_only(fn, prec):
    for n in (1, 2, 16, 33, 64, 256, 512):
        c = cf.chessfad_default_config(fn, n, 1000, prec)
        assert c.csize in (1, 2, 4, 8, 16, 32)
        assert c.csize <= max(1, 1 << (n - 1).bit_length())
        nch = -(-n // c.csize)
        assert 1 <= c.threads_per_row <= 32 and c.threads_per_row & (c.threads_per_row - 1) == 0
        assert c.threads_per_row <= max(1, 1 << (nch - 1).bit_length())
        assert c.block_threads % 32 == 0


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle (the oracle is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2410_22575_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f
