"""GPU test of the precision pattern on its own workload: the two merging
drops of Sec. 5.2 (256 x 128 periodic, R = 25, 2-cell gap, W = 5, density
ratio 5 with equal kinematic viscosities, sigma = 1e-3, M = 0.05) advanced
20000 steps with float32, FP16 and BF16 population storage, against the FP64
oracle from the same phi0, for each force family (STF-1, CPF-1, PF-1, CSF-1).

Reported for every storage format: the max-abs error of phi and u and the
error of the pressure jump Delta p (mean p_h within r <= 12 of the domain
centre minus the mean beyond r >= 50), relative to the Laplace jump sigma/R_m
of the merged drop (R_m = 25 sqrt 2; the oracle's Delta p passes through zero
while the drops merge), after 2000 steps and after 20000.

The merge amplifies rounding: the float32 path itself moves away from the
FP64 oracle as the bridge between the drops forms.  At 2000 steps its phi and
u errors must stay within 5x those of the oracle's own algorithm run with
float32 state (oracle.float32_deviation).  The other bars are the measured
errors with margin (GB300, every family; the largest measured value in
brackets): float32 phi 1e-3 [3.3e-4], u 3e-5 [1.05e-5], Delta p 1 %
[0.35 %]; FP16 phi 3e-2 [1.1e-2], u 1e-4 [4.5e-5], Delta p 3 % [0.86 %];
BF16 phi 0.3 [0.15], u 3e-4 [7.6e-5], Delta p 10 % [5.0 %, at 2000 steps].
BF16's 8-bit mantissa keeps the merged drop within a fraction of a cell of
the FP64 one, but not at the 1e-3 level over 20000 steps."""
import numpy as np
import pytest

from paper_2012_14729_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FAMILIES = ("STF1", "CPF1", "PF1", "CSF1")
STEPS = (2000, 20000)
R_IN, R_OUT = 12.0, 50.0
BARS = {"fp32": (1e-3, 3e-5, 0.01), "fp16": (3e-2, 1e-4, 0.03), "bf16": (0.3, 3e-4, 0.10)}


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_14729_gb300 import build, pflbm
    build.build()
    pflbm.load()
    return pflbm


def _dp(fields, nx, ny):
    Y, X = np.mgrid[0:ny, 0:nx].astype(float)
    r = np.hypot(X - nx / 2, Y - ny / 2)
    ph = fields["p_h"].astype(np.float64)
    return float(ph[r <= R_IN].mean() - ph[r >= R_OUT].mean())


@pytest.fixture(scope="module")
def oracle_runs(orc):
    """FP64 oracle fields at each checkpoint, per form (run once)."""
    out = {}
    for form in FAMILIES:
        c = wl.merging_drops(form)
        s = orc.Sim(c.nx, c.ny, c.wall_y, orc.Params(**c.params),
                    c.phi0.astype(np.float32).astype(np.float64))
        done, res = 0, {}
        for T in STEPS:
            s.step(T - done)
            done = T
            res[T] = s.macro()
        # float32 rounding sensitivity over the first checkpoint
        dev = orc.float32_deviation(c.nx, c.ny, c.wall_y, orc.Params(**c.params),
                                    c.phi0.astype(np.float32).astype(np.float64), STEPS[0])
        out[form] = (c, res, dev)
    return out


@pytest.mark.parametrize("form", FAMILIES)
def test_merging_drops_16bit_storage_against_fp64(pf, oracle_runs, form):
    c, ref, dev = oracle_runs[form]
    lines, fails = [], []
    for storage in ("fp32", "fp16", "bf16"):
        d = pf.Domain(c.nx, c.ny, wall_y=False, storage=storage).set_params(**c.params)
        d.init_phi(c.phi0.astype(np.float32))
        done = 0
        for T in STEPS:
            d.step(T - done)
            done = T
            g = d.fields()
            o = ref[T]
            e_phi = float(np.abs(g["phi"] - o["phi"]).max())
            e_u = float(max(np.abs(g["ux"] - o["ux"]).max(), np.abs(g["uy"] - o["uy"]).max()))
            dp_o = _dp(o, c.nx, c.ny)
            laplace = c.params["sigma"] / (c.meta["R"] * np.sqrt(2.0))
            e_dp = abs(_dp(g, c.nx, c.ny) - dp_o) / laplace
            lines.append(f"{storage} t={T}: phi {e_phi:.2e} u {e_u:.2e} dp {e_dp:.2e} "
                         f"(oracle dp {dp_o:.4e})")
            b_phi, b_u, b_dp = BARS[storage]
            if storage == "fp32" and T == STEPS[0]:
                b_phi, b_u = max(1e-5, 5 * dev["phi"]), max(1e-6, 5 * dev["u"])
                lines[-1] += f" [float32 state: phi {dev['phi']:.2e} u {dev['u']:.2e}]"
            if not (e_phi <= b_phi and e_u <= b_u and e_dp <= b_dp):
                fails.append(lines[-1])
    print(f"PRECISION {form}: " + "; ".join(lines))
    assert not fails, fails
