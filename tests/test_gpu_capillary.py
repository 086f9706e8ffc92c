"""Capillary wave (Sec. 5.3) on the GPU against the analytic amplitude
(Prosperetti's solution): H = 80, Re = 50, We = 1, density ratio 1 and 10,
every force form, over the paper's error window [0, 25/omega_0], with E_2 of
Eq. capilary_error set beside the paper's table (tests/golden/
capillary_table.json).  Measured: ratio 1, 1.06x (CSF-2) to 2.0x (CPF-1) the
paper's E_2 with the same extremes (CSF-2 best, PF-2 worst); ratio 10,
0.15-0.19 against the paper's 0.026-0.038.  The same run against the FP64
oracle: the state after 2000 steps element by element, and the amplitude
series and E_2 over the whole window."""
import json
import os

import numpy as np
import pytest

from paper_2012_14729_gb300 import validation as v
from paper_2012_14729_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FORMS = ("STF1", "STF2", "CPF1", "CPF2", "PF1", "PF2", "CSF1", "CSF2")
# at density ratio 10 these forms diverge within 2000 steps, in the FP64
# oracle as on the GPU (a property of the scheme at these parameters)
DIVERGE_AT_10 = ("CPF1", "PF2", "CSF2")
TABLE = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                    "capillary_table.json")))["E2"]


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_14729_gb300 import build, pflbm
    build.build()
    pflbm.load()
    return pflbm


@pytest.mark.parametrize("ratio", [1.0, 10.0])
@pytest.mark.parametrize("form", FORMS)
def test_capillary_wave_follows_the_analytic_amplitude(pf, form, ratio):
    if ratio == 10.0 and form in DIVERGE_AT_10:
        pytest.skip("diverges at density ratio 10 in the FP64 oracle too")
    case = wl.capillary_wave(form, H=80, rho_ratio=ratio)
    t, h, th, e2 = v.run_capillary_wave(pf, case, every=90)
    paper = TABLE[f"{ratio:g}"]["H80"][form]
    print(f"CAP {form} ratio {ratio:g}: E2 = {e2:.4f} (paper {paper}); h/h0 every 900 steps "
          f"{np.round(h[::10], 3).tolist()} theory {np.round(th[::10], 3).tolist()}")
    assert np.all(np.isfinite(h))
    if ratio == 1.0:
        assert e2 <= 2.5 * paper, (e2, paper)   # measured up to 2.0x
    else:
        assert e2 <= 0.25, (e2, paper)          # measured 0.15-0.19
    # the first half period follows the analytic solution closely
    first = t <= np.pi / np.sqrt(case.params["sigma"] * case.meta["k"] ** 3 /
                                 (case.params["rho1"] + case.params["rho2"]))
    assert np.abs(h[first] - th[first]).max() <= 0.25  # measured 0.03-0.18


@pytest.mark.parametrize("form", ["STF1", "CSF2"])
def test_capillary_wave_matches_oracle(pf, orc, form):
    """H = 80, density ratio 1.  After 2000 steps: phi and u element by element
    at the fixed bar (1e-5, 1e-6) or 5x the deviation of the oracle's own
    algorithm with float32 state, whichever is larger (the tolerance used is
    printed).  Over [0, 25/omega_0]: the amplitude h(t)/h0 sampled every 900
    steps within 3e-3 of the oracle's (measured 7e-5 for STF-1, 1.4e-3 for
    CSF-2) and E_2 within 1 % of it (measured 0.02 % and 0.6 %)."""
    case = wl.capillary_wave(form, H=80, rho_ratio=1.0)
    phi0 = case.phi0.astype(np.float32)
    par = orc.Params(**case.params)
    d = pf.Domain(case.nx, case.ny, wall_y=True).set_params(**case.params).init_phi(phi0)
    d.step(2000)
    g = d.fields()
    dev = orc.float32_deviation(case.nx, case.ny, True, par, phi0.astype(np.float64), 2000)
    o = dev["fields64"]
    e_phi = float(np.abs(g["phi"] - o["phi"]).max())
    e_u = float(max(np.abs(g["ux"] - o["ux"]).max(), np.abs(g["uy"] - o["uy"]).max()))
    tol_phi, tol_u = max(1e-5, 5 * dev["phi"]), max(1e-6, 5 * dev["u"])
    print(f"CAP-ORACLE {form} t=2000: phi {e_phi:.2e} (tol {tol_phi:.2e}, float32 state "
          f"{dev['phi']:.2e}), u {e_u:.2e} (tol {tol_u:.2e})")
    assert e_phi <= tol_phi and e_u <= tol_u

    every = 900
    t, h, th, e2 = v.run_capillary_wave(pf, case, every=every)
    s = orc.Sim(case.nx, case.ny, True, par, phi0.astype(np.float64))
    ho = [v.wave_amplitude(s.macro()["phi"]) / case.meta["h0"]]
    for _ in range(len(t) - 1):
        s.step(every)
        ho.append(v.wave_amplitude(s.macro()["phi"]) / case.meta["h0"])
    ho = np.asarray(ho)
    e2o = v.time_averaged_error(t, ho, th)
    print(f"CAP-ORACLE {form}: E2 GPU {e2:.5f} oracle {e2o:.5f}; max |h - h_oracle| / h0 "
          f"{np.abs(h - ho).max():.2e}")
    assert np.abs(h - ho).max() <= 3e-3
    assert abs(e2 - e2o) <= 0.01 * e2o
