"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/pflbm.h declares, and its host-side argument checks
behave as documented (no GPU call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pflbm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(pflbm_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2012_14729_gb300 import build, pflbm
    build.build()
    return pflbm.load()


def test_header_declares_api():
    names = declared_functions()
    for must in ("pflbm_create", "pflbm_set_params", "pflbm_init_phi", "pflbm_step",
                 "pflbm_read", "pflbm_diagnostics", "pflbm_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2012_14729_gb300 import pflbm
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in pflbm.SIGNATURES, f"binding lacks {name}"


def test_workspace_bytes(lib):
    from paper_2012_14729_gb300 import pflbm
    assert pflbm.pflbm_workspace_bytes(3, 64, 0) == 0
    assert pflbm.pflbm_workspace_bytes(64, 3, 0) == 0
    n32 = pflbm.pflbm_workspace_bytes(64, 64, 0)
    n16 = pflbm.pflbm_workspace_bytes(64, 64, 1)
    # two FP32 population buffers of 18 planes of (ny + 2) x nx
    assert n32 >= 2 * 18 * 66 * 64 * 4
    assert n16 < n32
    assert n32 % 256 == 0


def test_create_and_param_checks(lib):
    from paper_2012_14729_gb300 import pflbm
    fake = 1 << 20  # aligned placeholder address: create and set_params never touch it
    nbytes = pflbm.pflbm_workspace_bytes(16, 16, 0)
    with pytest.raises(pflbm.PflbmError) as e:
        pflbm.pflbm_create(16, 16, 1, 0, 0, fake, nbytes, None)  # x walls unsupported
    assert e.value.status == 1
    with pytest.raises(pflbm.PflbmError) as e:
        pflbm.pflbm_create(16, 16, 0, 0, 0, fake, nbytes - 256, None)
    assert e.value.status == 2
    with pytest.raises(pflbm.PflbmError):
        pflbm.pflbm_create(16, 16, 0, 0, 0, fake + 8, nbytes, None)  # misaligned
    d = pflbm.pflbm_create(16, 16, 0, 1, 0, fake, nbytes, None)
    try:
        pflbm.pflbm_set_params(d, pflbm.make_params())
        for bad in (dict(tau_h=0.5), dict(W=0.0), dict(M=-1.0), dict(rho2=0.0),
                    dict(nu1=0.0), dict(form=8), dict(scale_f=3.0), dict(eps=-1.0)):
            with pytest.raises(pflbm.PflbmError) as e:
                pflbm.pflbm_set_params(d, pflbm.make_params(**bad))
            assert e.value.status == 1
        # stepping before an initial state is an ordering error
        with pytest.raises(pflbm.PflbmError) as e:
            pflbm.pflbm_step(d, 1)
        assert e.value.status == 6
    finally:
        pflbm.pflbm_destroy(d)


def test_status_strings(lib):
    assert lib.pflbm_status_str(0) == b"ok"
    assert b"sm_103a" in lib.pflbm_version()


def test_noalloc_diagnostics_size_checks(lib):
    """The no-allocation diagnostics reject sizes before any CUDA call."""
    from paper_2012_14729_gb300 import pflbm
    fake = 1 << 20  # never dereferenced: the size checks come first
    out = pflbm.pflbm_diag()
    f = lib.pflbm_field_diagnostics_noalloc
    assert f(0, 16, 0, 0, fake, None, ctypes.byref(out), None) == 1
    assert f(16, -1, 0, 0, fake, None, ctypes.byref(out), None) == 1
    assert f(16, 16, 0, 0, fake, None, None, None) == 1
    # boundary kinds: x periodic or free-slip, y periodic or wall
    assert f(16, 16, pflbm.WALL, 0, fake, None, ctypes.byref(out), None) == 1
    assert f(16, 16, 0, pflbm.FREESLIP, fake, None, ctypes.byref(out), None) == 1
    assert "bc_x must be" in lib.pflbm_last_error().decode()
    assert pflbm.NOALLOC_MAX_NODES == 4096 * 2048
    assert f(4096, 2049, 0, 0, fake, None, ctypes.byref(out), None) == 1
    msg = lib.pflbm_last_error().decode()
    assert "8392704 nodes" in msg and "at most 8388608 nodes" in msg
    hdr = open(HEADER).read()
    assert re.search(r"#define PFLBM_NOALLOC_MAX_NODES\s+%d\b" % pflbm.NOALLOC_MAX_NODES, hdr)


def test_size_limits_of_32_bit_plane_offsets(lib):
    """Sizes whose plane offsets would not fit 32 bits are refused on the
    host: the population planes (9 (ny + 2) nx < 2^31) and the adjoint's tape
    (24 nx ny < 2^31).  No CUDA call: create never touches the workspace."""
    from paper_2012_14729_gb300 import pflbm
    assert pflbm.pflbm_workspace_bytes(16384, 14560, 0) > 0      # 9 * 14562 * 16384 < 2^31
    assert pflbm.pflbm_workspace_bytes(16384, 14564, 0) == 0     # >= 2^31
    assert pflbm.pflbm_workspace_bytes(14564, 16384, 1) == 0
    fake = 1 << 20
    for ny, ok in ((5461, True), (5462, False)):                 # 24 * 16384 * ny vs 2^31
        nbytes = pflbm.pflbm_workspace_bytes(16384, ny, 0)
        d = pflbm.pflbm_create(16384, ny, 0, 1, 0, fake, nbytes, None)
        try:
            got = lib.pflbm_adjoint_scratch_bytes(d, 10, 5)
            assert (got > 0) == ok, (ny, got)
        finally:
            pflbm.pflbm_destroy(d)
