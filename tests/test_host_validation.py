"""Host-side argument validation of the C ABI, on a CPU-only host: every call here is rejected
(or answered) before any CUDA call is made, so no GPU is needed.

The FFT sides follow the rule stated in include/zm.h: low and medium order take periodic sides
R 2^a (a >= 3, R odd 1 .. 19, side <= 8192); the double-word path the same except powers of two
above 4096.
"""
import pytest

from paper_2406_05490_gb300 import build


@pytest.fixture(scope="module")
def zm():
    build.build()
    from paper_2406_05490_gb300 import zm as _zm
    _zm._lib = None
    _zm.load()
    return _zm


def code_of(zm, fn):
    with pytest.raises(zm.ZMError) as e:
        fn()
    return e.value.code


@pytest.mark.parametrize("n1,n2,order_name,prec_name,periodic,delta,expect", [
    (4, 32, "HIGH", None, True, 0.01, "INVALID"),            # sides >= 5
    (32, 32, "HIGH", None, True, 0.0, "INVALID"),            # delta > 0 for the all-pairs sum
    (32, 32, "MEDIUM", None, True, 0.0, "INVALID"),
    (32, 32, "LOW", None, False, None, "UNSUPPORTED"),       # the FFT needs a periodic mesh
    (32, 32, "MEDIUM", None, False, 0.01, "UNSUPPORTED"),
    (12, 16, "LOW", None, True, None, "UNSUPPORTED"),        # 12 = 3 x 2^2: a < 3
    (168, 64, "LOW", None, True, None, "UNSUPPORTED"),       # 168 = 21 x 2^3: R > 19
    (64, 44, "LOW", None, True, None, "UNSUPPORTED"),        # 44 = 11 x 2^2
    (16384, 8, "LOW", None, True, None, "UNSUPPORTED"),      # above 8192
    (8192, 8, "LOW", "DF64", True, None, "UNSUPPORTED"),     # double words: powers of two <= 4096
    (32, 32, "HIGH", "DF64", True, 0.01, "UNSUPPORTED"),     # double words: low order only
    (32, 32, "LOW", "DF64|FP32C", True, None, "INVALID"),    # two precisions
    (8193, 8192, "HIGH", None, True, 0.01, "INVALID"),       # n1 n2 <= 2^26
])
def test_create_rejects(zm, n1, n2, order_name, prec_name, periodic, delta, expect):
    order = getattr(zm, f"ZM_ORDER_{order_name}")
    for p in (prec_name or "").split("|"):
        if p:
            order |= getattr(zm, f"ZM_PREC_{p}")
    code = code_of(zm, lambda: zm.zm_create(n1, n2, periodic=periodic, order=order, delta=delta))
    assert code == getattr(zm, f"ZM_ERR_{expect}")


def test_request_bytes_and_strings(zm):
    # the server's admission size of one interface: proportional to the node count once the
    # padding of the last tiles (records sized for every candidate tile shape) is small
    b256, b512 = zm.zm_server_request_bytes(256, 256), zm.zm_server_request_bytes(512, 512)
    assert 0 < zm.zm_server_request_bytes(32, 32) < b256 < b512 and 3.9 < b512 / b256 < 4.1
    assert code_of(zm, lambda: zm.zm_server_request_bytes(4, 4)) == zm.ZM_ERR_INVALID
    lib = zm.load()
    for code in range(0, -8, -1):
        assert lib.zm_error_string(code)
    assert zm.zm_checked_build() is False


def test_noalloc_rejects_on_the_host(zm):
    """The allocation-free sum refuses, before any CUDA work: n outside [1, 65536], buffers
    shorter than 3 n (binding), and, with no GPU, any pointer (none is device memory)."""
    import numpy as np
    a = np.zeros((3, 8))
    assert code_of(zm, lambda: zm.zm_br_velocity_noalloc(65537, a, a, 0.01, a)) == zm.ZM_ERR_INVALID
    assert code_of(zm, lambda: zm.zm_br_velocity_noalloc(0, a, a, 0.01, a)) == zm.ZM_ERR_INVALID
    assert code_of(zm, lambda: zm.zm_br_velocity_noalloc(9, a, a, 0.01, a)) == zm.ZM_ERR_INVALID
    assert code_of(zm, lambda: zm.zm_br_velocity_noalloc(8, a, a, 0.0, a)) == zm.ZM_ERR_INVALID
    assert code_of(zm, lambda: zm.zm_br_velocity_noalloc(8, a, a, 0.01, a)) == zm.ZM_ERR_INVALID
