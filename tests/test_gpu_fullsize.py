"""Parity at the benchmark's full sizes, in the launch configurations the
benchmark times, on sampled outputs the oracle computes patch by patch.

The GPU advances the 512 x 1024 rising-bubble workload (walls at bottom and
top, density ratio 10, seeded noise) and the 2048 x 4096 side-wall rising
bubble; one more GPU step is then checked against the FP64 oracle on square
patches.  Each patch starts from the GPU's own state (pre-collision f and h
read back, and phi u of the previous step from the fields read one step
earlier), takes one oracle step with the patch's edges periodic, and its
populations are compared where the step cannot see those edges: a node's
new pre-collision value depends on the old state within 4 nodes (phi on the
3-ring of the force stencils, then the pull), so a 5-node band is left out.
Patches at the bottom and top walls keep the wall (the oracle's patch has
walls at both ends and the far band is left out), and one patch straddles
the periodic seam in x."""
import numpy as np
import pytest

from paper_2012_14729_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

P, M = 40, 5          # patch side, excluded band
TOL = 1e-5            # of each population family's largest value in the patch


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_14729_gb300 import build, pflbm
    build.build()
    pflbm.load()
    return pflbm


def _gpu_rho0(p, phi0):
    # the library's default: rho(mean phi0), mean over the float32 phi0 in
    # double, rounded to float32
    m = float(phi0.astype(np.float32).astype(np.float64).mean())
    return float(np.float32(0.5 * p["rho1"] * (1 + m) + 0.5 * p["rho2"] * (1 - m)))


def _run(pf, case, stage, steps, wall_x):
    d = pf.Domain(case.nx, case.ny, wall_y=True, wall_x=wall_x).set_params(**case.params)
    d.stage_mode(stage)
    d.init_phi(case.phi0.astype(np.float32))
    d.step(steps)
    fl = d.fields()
    phiu_prev = np.stack([fl["phi"] * fl["ux"], fl["phi"] * fl["uy"]])  # float32 products
    d.step(1)
    f1, h1 = d.populations()
    d.step(1)
    f2, h2 = d.populations()
    return phiu_prev, (f1, h1), (f2, h2)


def _patch(a, y0, x0):
    nx = a.shape[-1]
    cols = np.arange(x0, x0 + P) % nx
    return np.ascontiguousarray(a[..., y0:y0 + P, :][..., cols].astype(np.float64))


def _check_patches(orc, case, state, patches, wall_x_patch=False):
    phiu_prev, (f1, h1), (f2, h2) = state
    p = dict(case.params)
    p["rho0"] = _gpu_rho0(p, case.phi0)
    par = orc.Params(**p)
    worst = 0.0
    for y0, x0, where in patches:
        s = orc.Sim(P, P, True, par, np.zeros((P, P)))
        s.f = _patch(f1, y0, x0)
        s.h = _patch(h1, y0, x0)
        s.phiu_prev = _patch(phiu_prev, y0, x0)
        s.t = 1  # not the first step of a run
        s.step(1)
        ylo = 0 if where == "bottom" else M
        yhi = P if where == "top" else P - M
        sl = (slice(None), slice(ylo, yhi), slice(M, P - M))
        for name, o, g in (("f", s.f, _patch(f2, y0, x0)), ("h", s.h, _patch(h2, y0, x0))):
            err = float(np.abs(o[sl] - g[sl]).max())
            scale = float(np.abs(g[sl]).max())
            worst = max(worst, err / scale)
            assert err <= TOL * scale + 1e-12, (where, y0, x0, name, err, scale)
    return worst


@pytest.mark.parametrize("stage", ["gather", "boxes"])
def test_bench_workload_512x1024_sampled(pf, orc, stage):
    c = wl.capillary_bubble("bubble")
    state = _run(pf, c, stage, 40, False)
    rng = np.random.default_rng(7)
    patches = [(int(rng.integers(8, c.ny - P - 8)), int(rng.integers(0, c.nx)), "interior")
               for _ in range(4)]
    patches += [(0, 100, "bottom"), (c.ny - P, 300, "top"), (500, c.nx - P // 2, "seam"),
                (c.ny // 4 - P // 2, c.nx // 2 - P // 2, "interface")]
    worst = _check_patches(orc, c, state, patches)
    print(f"{stage}: largest error / scale {worst:.2e}")


def test_side_wall_workload_2048x4096_sampled(pf, orc):
    c = wl.rising_bubble("STF1", nx=2048)
    state = _run(pf, c, "gather", 20, True)
    R = int(c.meta["R"])
    yc = xc = c.nx // 2
    # interior patches on the bubble's interface and in the bulk
    patches = [(yc - R - P // 2, xc - P // 2, "interior"), (yc - P // 2, xc + R - P // 2, "interior"),
               (3000, 1000, "interior"), (0, 700, "bottom"), (c.ny - P, 1500, "top")]
    _check_patches(orc, c, state, patches)
