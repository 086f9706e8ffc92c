"""GPU test of pflbm_field_diagnostics_noalloc, the FP64 diagnostics that
run on the library's static scratch array instead of workspace memory.

Two calls in a row on the same fields give the same result bit for bit and
agree with pflbm_diagnostics (workspace scratch) to FP64 summation order; a
call on a larger lattice followed by one on a smaller leaves nothing stale.
This file is collected last so that it also runs after every other test has
used the library in the same process."""
import numpy as np
import pytest

from paper_2012_14729_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

KEYS = ("mass", "umax", "area1", "R_num", "p_in", "p_out", "dp", "sigma_num", "xc1", "yc1",
        "taylor_D", "nonfinite")


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_14729_gb300 import build, pflbm
    build.build()
    pflbm.load()
    return pflbm


def _run(pf, nx, ny, steps):
    """A drop advanced `steps` steps; its fields on the device, the geometry
    of the pressure jump and pflbm_diagnostics of the same state."""
    import torch
    r = min(nx, ny) / 5
    phi0 = wl.drop(nx, ny, r, 4.0, xc=nx / 2 - 0.3, yc=ny / 2 + 0.2)
    d = pf.Domain(nx, ny, wall_y=False).set_params(sigma=0.01, W=4.0, M=0.1, rho1=1.0,
                                                   rho2=0.1, nu1=0.1, nu2=0.1, form="STF1")
    d.init_phi(phi0)
    d.step(steps)
    fields = torch.empty((len(pf.FIELDS), ny, nx), dtype=torch.float32, device="cuda")
    pf.pflbm_read_fields(d.h, fields)
    d.synchronize()
    geom = pf.pflbm_diag_geom(nx / 2, ny / 2, 0.5 * r, 1.5 * r)
    st, ref = pf.pflbm_diagnostics(d.h, geom)
    assert st == 0
    return d, fields, geom, ref.as_dict()


def _noalloc(pf, d, fields, geom):
    ny, nx = fields.shape[1:]
    st, out = pf.pflbm_field_diagnostics_noalloc(nx, ny, fields, geom, d.stream)
    return st, out.as_dict()


def _close(a, b):
    for k in KEYS:
        assert abs(a[k] - b[k]) <= 1e-12 * abs(b[k]) + 1e-15, (k, a[k], b[k])


def test_two_calls_in_a_row_match_workspace_diagnostics(pf):
    # 200 x 150 = 30000 nodes: 118 blocks, the last one ragged
    d, fields, geom, ref = _run(pf, 200, 150, 40)
    st1, a = _noalloc(pf, d, fields, geom)
    st2, b = _noalloc(pf, d, fields, geom)
    assert st1 == 0 and st2 == 0
    assert a == b
    _close(a, ref)
    assert ref["p_in"] != 0.0 and ref["umax"] > 0.0


def test_larger_then_smaller_lattice(pf):
    # 1024 x 600 nodes take more partial rows (600 blocks) than the workspace
    # reduction's 1024-block grid-stride layout, so the two orders differ
    big = _run(pf, 1024, 600, 10)
    small = _run(pf, 96, 40, 10)
    st, a = _noalloc(pf, *big[:3])
    assert st == 0
    _close(a, big[3])
    st, b = _noalloc(pf, *small[:3])
    assert st == 0
    _close(b, small[3])
    st, c = _noalloc(pf, *small[:3])
    assert st == 0 and c == b


def test_nonfinite_node_and_host_pointer(pf):
    import torch
    d, fields, geom, ref = _run(pf, 64, 48, 5)
    bad = fields.clone()
    bad[0, 7, 9] = float("nan")
    torch.cuda.synchronize()  # written on torch's stream, read on the domain's
    ny, nx = fields.shape[1:]
    st, out = pf.pflbm_field_diagnostics_noalloc(nx, ny, bad, geom, d.stream)
    assert st == 4 and out.nonfinite == 1.0
    # a host array is refused before any launch
    host = np.zeros((len(pf.FIELDS), ny, nx), np.float32)
    with pytest.raises(pf.PflbmError) as e:
        pf.pflbm_field_diagnostics_noalloc(nx, ny, host, geom, d.stream)
    assert e.value.status == 1 and "device memory" in str(e.value)
    # and the scratch still gives the right answer afterwards
    st, out = _noalloc(pf, d, fields, geom)
    assert st == 0
    _close(out, ref)
