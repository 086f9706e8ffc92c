"""The rising-bubble benchmark of Sec. 5.4 on the GPU: free-slip side walls,
no-slip top and bottom, density and viscosity ratio 10, Re = 35, Eo = 10,
120 x 240 nodes, every force form run to t = 3 s with the centre of mass,
rise velocity and circularity sampled through pflbm_bubble_diagnostics.

Checked: the run stays finite; the mirror symmetry of the problem about the
vertical midline holds (x-centroid on the midline); the centre of mass rises
monotonically; and the paper's benchmark quantities fall in sanity bands
around its printed values (Table rising, tests/golden/rising_bubble_table.json:
y_c max 1.0536-1.0681 m, v_c max 0.2223-0.2284 m/s, circularity min
0.8889-0.9004 at 240 x 480).  Measured
here: STF/CPF/PF forms v_max 0.195-0.199 m/s, y_c(3 s) 0.971-0.985 m,
C_min 0.955-0.962; CSF-1 0.217 / 1.077 / 0.962; CSF-2 0.236 / 1.067 / 0.894.
These are bands, not parity: the paper does not give its mobility or
interface width (the workload's choices are those every form is stable
with), and the parity of the quantities themselves is tested against the
oracle in test_gpu_bubble.py."""
import json
import os

import numpy as np
import pytest

from paper_2012_14729_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FORMS = ("STF1", "STF2", "CPF1", "CPF2", "PF1", "PF2", "CSF1", "CSF2")
TABLE = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                    "rising_bubble_table.json")))


def _band(key, lo, hi):
    """[lo x the smallest printed value over the forms, hi x the reference]."""
    vals = [v[key] for v in TABLE["forms"].values()]
    return lo * min(vals), hi * TABLE["reference"][key]


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_14729_gb300 import build, pflbm
    build.build()
    pflbm.load()
    return pflbm


# (nx, settings): the workload's defaults on 120 x 240; on the paper's finer
# 240 x 480 grid the setting of the same width W = 8 that every form but
# CPF-1 runs to 3 s with (CPF-1 diverges there: the FP64 oracle between
# steps 7400 and 7600, the GPU by step 7224)
GRIDS = {120: {}, 240: dict(Ug=0.02, W=8.0, M=0.1, tau_h=0.8)}


@pytest.mark.parametrize("nx", [120, 240])
@pytest.mark.parametrize("form", FORMS)
def test_rising_bubble_to_three_seconds(pf, form, nx):
    if nx == 240 and form == "CPF1":
        pytest.skip("CPF-1 diverges on 240 x 480 with these settings")
    c = wl.rising_bubble(form, nx=nx, **GRIDS[nx])
    d = pf.Domain(c.nx, c.ny, wall_y=True, wall_x=True).set_params(**c.params)
    d.init_phi(c.phi0.astype(np.float32))
    m = c.meta
    nsteps = int(round(3.0 / m["s_per_step"]))
    every = nsteps // 150
    mid = 0.5 * c.nx - 0.5
    tol_mid = 2e-3 * c.nx / 120
    t, yc, vc, C = [], [], [], []
    n = 0
    while n < nsteps:
        k = min(every, nsteps - n)
        d.step(k)
        n += k
        g = d.bubble_diagnostics()
        assert g["status"] == "PFLBM_OK", (form, n)
        # mirror symmetry about the midline, up to float32 rounding order
        assert abs(g["xc2"] - mid) < tol_mid, (form, n, g["xc2"])
        t.append(n * m["s_per_step"])
        yc.append((g["yc2"] + 0.5) * m["m_per_node"])
        vc.append(g["vc2"] * m["mps_per_lattice"])
        C.append(g["circularity"])
    assert t[-1] == pytest.approx(3.0, abs=m["s_per_step"])
    assert np.all(np.diff(yc) >= -1e-6), form
    # bands: v_max [0.178, 0.266], C_min [0.844, 0.982], y_max [0.948, 1.125]
    lo, hi = _band("v_max", 0.8, 1.1)
    assert lo <= max(vc) <= hi, (form, max(vc))
    lo, hi = _band("C_min", 0.95, 1.09)
    assert lo <= min(C) <= hi, (form, min(C))
    lo, hi = _band("y_max", 0.9, 1.04)
    assert lo <= max(yc) <= hi, (form, max(yc))
    # the bubble starts round and at rest
    assert C[0] == pytest.approx(1.0, abs=5e-3) and abs(vc[0]) < 0.02
