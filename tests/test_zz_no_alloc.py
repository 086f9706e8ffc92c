"""GPU test of pflbm_field_diagnostics_noalloc, the FP64 diagnostics that
run on the library's static scratch array instead of workspace memory.

Two calls in a row on the same fields give the same result bit for bit and
agree with pflbm_diagnostics (workspace scratch) to FP64 summation order; a
call on a larger lattice followed by one on a smaller leaves nothing stale; on
a lattice with walls the pressure-jump distance does not wrap across them; a
call after the first leaves the device's free memory unchanged; the largest
accepted lattice (every partial row of the array in use) matches FP64 sums
taken by torch.  This file is collected last so that it also runs after every
other test has used the library in the same process."""
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


def _run(pf, nx, ny, steps, walls=False, centre=None):
    """A drop advanced `steps` steps; its fields on the device, the geometry
    of the pressure jump and pflbm_diagnostics of the same state.  walls:
    no-slip walls in y and free-slip walls in x."""
    import torch
    r = min(nx, ny) / 5
    xc, yc = centre if centre else (nx / 2 - 0.3, ny / 2 + 0.2)
    phi0 = wl.drop(nx, ny, r, 4.0, xc=xc, yc=yc, periodic_y=not walls)
    d = pf.Domain(nx, ny, wall_y=walls, wall_x=walls).set_params(
        sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.1, nu1=0.1, nu2=0.1, form="STF1")
    d.init_phi(phi0)
    d.step(steps)
    fields = torch.empty((len(pf.FIELDS), ny, nx), dtype=torch.float32, device="cuda")
    pf.pflbm_read_fields(d.h, fields)
    d.synchronize()
    geom = pf.pflbm_diag_geom(xc, yc, 0.5 * r, 1.5 * r)
    st, ref = pf.pflbm_diagnostics(d.h, geom)
    assert st == 0
    d.walls = walls
    return d, fields, geom, ref.as_dict()


def _bc(pf, d):
    walls = getattr(d, "walls", False)
    return (pf.FREESLIP if walls else pf.PERIODIC), (pf.WALL if walls else pf.PERIODIC)


def _noalloc(pf, d, fields, geom):
    ny, nx = fields.shape[1:]
    bx, by = _bc(pf, d)
    st, out = pf.pflbm_field_diagnostics_noalloc(nx, ny, fields, geom, d.stream, bx, by)
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


def test_walls_do_not_wrap_the_pressure_jump_distance(pf):
    """An off-centre drop next to the bottom wall of a lattice with no-slip
    walls in y and free-slip walls in x: nodes by the top wall are far from the
    drop, not (periodically) close to it."""
    d, fields, geom, ref = _run(pf, 120, 90, 30, walls=True, centre=(30.0, 20.0))
    st, a = _noalloc(pf, d, fields, geom)
    assert st == 0
    _close(a, ref)
    # FP64 means over the same float32 fields with the plain distance
    f = fields.double().cpu().numpy()
    ph = f[6]
    Y, X = np.mgrid[0:90, 0:120].astype(float)
    r = np.hypot(X - geom.xc, Y - geom.yc)
    p_in, p_out = ph[r <= geom.r_in].mean(), ph[r >= geom.r_out].mean()
    assert a["p_in"] == pytest.approx(p_in, rel=1e-12, abs=1e-15)
    assert a["p_out"] == pytest.approx(p_out, rel=1e-12, abs=1e-15)
    # taking both sides as periodic counts other nodes outside
    st, wrapped = pf.pflbm_field_diagnostics_noalloc(120, 90, fields, geom, d.stream)
    assert st == 0 and wrapped.p_out != a["p_out"]


def test_calls_after_the_first_leave_free_memory_unchanged(pf):
    import torch
    d, fields, geom, ref = _run(pf, 96, 64, 5)
    st, _ = _noalloc(pf, d, fields, geom)  # loads the module if it was not yet
    assert st == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        st, out = _noalloc(pf, d, fields, geom)
        assert st == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    _close(out, ref)


def test_largest_lattice(pf):
    """4096 x 2048 = PFLBM_NOALLOC_MAX_NODES: every partial row of the array
    and the counter beside them in use; checked against FP64 sums by torch on
    the same float32 fields; one node more is refused."""
    import torch
    nx, ny = 4096, 2048
    assert nx * ny == pf.NOALLOC_MAX_NODES
    g = torch.Generator(device="cuda").manual_seed(5)
    fields = torch.rand((len(pf.FIELDS), ny, nx), generator=g, device="cuda") * 0.02 - 0.01
    yy = torch.arange(ny, device="cuda", dtype=torch.float64)[:, None]
    xx = torch.arange(nx, device="cuda", dtype=torch.float64)[None, :]
    rr = torch.hypot(xx - 1500.3, yy - 700.6)
    fields[0] = torch.tanh((300.0 - rr) / 2.0).float()
    torch.cuda.synchronize()
    geom = pf.pflbm_diag_geom(1500.3, 700.6, 150.0, 450.0)
    for _ in range(2):
        st, out = pf.pflbm_field_diagnostics_noalloc(nx, ny, fields, geom, None)
        assert st == 0
        o = out.as_dict()
        f = fields.double()
        phi = f[0]
        w = 0.5 * (1 + phi)
        m = float(w.sum())
        assert o["mass"] == pytest.approx(float(phi.sum()), rel=1e-11, abs=1e-8)
        assert o["area1"] == pytest.approx(m, rel=1e-12)
        assert o["xc1"] == pytest.approx(float((w * xx).sum()) / m, rel=1e-12)
        assert o["yc1"] == pytest.approx(float((w * yy).sum()) / m, rel=1e-12)
        assert o["umax"] == pytest.approx(float(torch.sqrt(f[2] ** 2 + f[3] ** 2).max()), rel=1e-12)
        dx = (xx - 1500.3).abs()
        dx = torch.minimum(dx, nx - dx)
        dy = (yy - 700.6).abs()
        dy = torch.minimum(dy, ny - dy)
        r = torch.sqrt(dx * dx + dy * dy)
        ph = f[6]
        assert o["p_in"] == pytest.approx(float(ph[r <= 150.0].mean()), rel=1e-9, abs=1e-14)
        assert o["p_out"] == pytest.approx(float(ph[r >= 450.0].mean()), rel=1e-9, abs=1e-14)
    with pytest.raises(pf.PflbmError) as e:
        pf.pflbm_field_diagnostics_noalloc(nx + 1, ny, fields, geom, None)
    assert e.value.status == 1 and "at most" in str(e.value)
