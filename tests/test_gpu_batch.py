"""GPU tests of the batched pattern: many domains of uneven sizes, force forms
and boundaries advanced by one persistent launch per step over a work-list of
(domain, tile) items, against the same domains stepped one by one and against
the FP64 oracle."""
import numpy as np
import pytest

from paper_2012_14729_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FORMS = ("STF1", "STF2", "CPF1", "CPF2", "PF1", "PF2", "CSF1", "CSF2")


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_14729_gb300 import build, pflbm
    build.build()
    pflbm.load()
    return pflbm


def _instances():
    """Eight instances: sizes 64^2 .. 160 x 96 (some ragged), every force
    form, walls on every third one, elliptic and circular drops."""
    out = []
    sizes = [(64, 64), (96, 80), (128, 128), (40, 72), (160, 96), (64, 48), (100, 100), (72, 136)]
    for k, (nx, ny) in enumerate(sizes):
        wall = k % 3 == 2
        R = 0.25 * min(nx, ny)
        phi0 = (wl.ellipse(nx, ny, R, 4.0, 0.1) if k % 2 else
                wl.drop(nx, ny, R, 4.0, periodic_y=not wall)).astype(np.float32)
        p = dict(sigma=10 ** (-4 + 2 * k / 7), W=4.0, M=0.1, rho1=1.0, rho2=0.5 if k % 2 else 1.0,
                 nu1=0.1, nu2=0.1, form=FORMS[k], uw_top=0.005 if wall else 0.0)
        out.append((nx, ny, wall, p, phi0))
    return out


def _domains(pf, insts, mode="gather", stream=None):
    doms = []
    for nx, ny, wall, p, phi0 in insts:
        d = pf.Domain(nx, ny, wall_y=wall, stream=stream).set_params(**p).stage_mode(mode)
        d.init_phi(phi0)
        doms.append(d)
    return doms


def _pops(doms):
    return [d.populations() for d in doms]


def _assert_close(a, b, tol_f=1e-9, tol_h=1e-6):
    for (fa, ha), (fb, hb) in zip(a, b):
        assert np.abs(fa - fb).max() <= tol_f
        assert np.abs(ha - hb).max() <= tol_h


def test_batch_equals_individual_steps(pf):
    insts = _instances()
    solo = _domains(pf, insts)
    for d in solo:
        d.step(30)
    doms = _domains(pf, insts)
    b = pf.Batch(doms)
    assert b.items == sum(((nx + 31) // 32) * ((ny + 15) // 16) for nx, ny, *_ in insts)
    b.step(30)
    b.synchronize()
    assert all(d.t == 30 for d in doms)
    _assert_close(_pops(doms), _pops(solo))


@pytest.mark.parametrize("mode,cps,rows", [("boxes", 2, 16), ("boxes", 1, 16), ("gather", 3, 16),
                                           ("gather", 1, 16), ("gather", 4, 8), ("gather", 2, 8)])
def test_batch_configs_agree(pf, mode, cps, rows):
    insts = _instances()
    ref = _domains(pf, insts)
    pf.Batch(ref).step(12).synchronize()
    doms = _domains(pf, insts)
    b = pf.Batch(doms).config(mode, cps, rows)
    assert b.tile_rows == rows
    assert b.items == sum(((nx + 31) // 32) * ((ny + rows - 1) // rows)
                          for nx, ny, *_ in insts)
    b.step(12)
    b.synchronize()
    _assert_close(_pops(doms), _pops(ref))


def test_batch_short_tiles_refuse_boxes(pf):
    doms = _domains(pf, _instances())
    b = pf.Batch(doms).config("gather", 4, 8)
    with pytest.raises(pf.PflbmError):
        pf.pflbm_batch_set_config(b.h, pf.STAGE_MODES["boxes"], 2)
    with pytest.raises(pf.PflbmError):
        pf.pflbm_batch_set_tile_rows(b.h, 12)
    b.config("boxes", 2)  # full tiles again, then boxes
    assert b.tile_rows == 16


def test_batch_graphs_equal_plain(pf):
    insts = _instances()
    a = _domains(pf, insts)
    pf.Batch(a).step(40).synchronize()
    c = _domains(pf, insts)
    bc = pf.Batch(c).graphs(True)
    bc.step(3)    # first steps, partly outside a graph
    bc.step(37)   # two graph replays of 16 plus a remainder
    bc.synchronize()
    for x, y in zip(_pops(a), _pops(c)):
        np.testing.assert_array_equal(x[0], y[0])
        np.testing.assert_array_equal(x[1], y[1])


def test_batch_instance_matches_oracle(pf, orc):
    insts = _instances()
    doms = _domains(pf, insts)
    pf.Batch(doms).step(200).synchronize()
    for k in (0, 2):  # a periodic and a walled instance
        nx, ny, wall, p, phi0 = insts[k]
        g = doms[k].fields()
        o = orc.Sim(nx, ny, wall, orc.Params(**p), phi0.astype(np.float64)).step(200).macro()
        e_phi = float(np.abs(g["phi"] - o["phi"]).max())
        e_u = float(max(np.abs(g["ux"] - o["ux"]).max(), np.abs(g["uy"] - o["uy"]).max()))
        assert e_phi <= 1e-5 and e_u <= 1e-6, (k, e_phi, e_u)


def test_batch_autotune_keeps_state(pf):
    insts = _instances()
    doms = _domains(pf, insts)
    b = pf.Batch(doms)
    b.step(3)
    b.synchronize()
    before = _pops(doms)
    mode, cps, rows = b.autotune(2)
    assert mode in ("boxes", "gather") and cps >= 1 and rows in (8, 16)
    assert rows == 16 or mode == "gather"
    after = _pops(doms)
    for x, y in zip(before, after):
        np.testing.assert_array_equal(x[0], y[0])
        np.testing.assert_array_equal(x[1], y[1])
    assert all(d.t == 3 for d in doms)
