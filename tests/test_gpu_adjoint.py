"""GPU tests of the hand-written adjoint (pattern 3): gradients of
J = sum (phi_T - phi_target)^2 with respect to sigma, M and the initial phi,
against central finite differences of the FP64 oracle (the FP64 reference
gradient) and of the float32 CUDA forward itself, for every force form with
periodic and walled boundaries, through checkpointed segments."""
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


def _case(wall, form):
    nx, ny = 24, 20
    phi0 = wl.drop(nx, ny, 6.0, 4.0, xc=11.7, yc=9.6, periodic_y=not wall)
    target = wl.drop(nx, ny, 6.5, 4.0, periodic_y=not wall)
    p = dict(sigma=0.02, W=4.0, M=0.1, rho1=1.0, rho2=0.5, nu1=0.1, nu2=0.05, gy=-1e-5,
             uw_bottom=-0.01 if wall else 0.0, uw_top=0.01 if wall else 0.0, form=form)
    # rho0 fixed (held constant by the adjoint)
    p["rho0"] = float(np.mean(0.5 * (1 + phi0) + 0.25 * (1 - phi0)))
    return nx, ny, phi0.astype(np.float32), target.astype(np.float32), p


def _gpu_adjoint(pf, nx, ny, wall, p, phi0, target, T, every):
    import torch
    d = pf.Domain(nx, ny, wall_y=wall).set_params(**p)
    dev = torch.device("cuda")
    phi0_t = torch.from_numpy(phi0).to(dev)
    # forward once for phi_T, then dJ/dphi_T
    d.init_phi(phi0_t)
    d.step(T)
    phiT = d.fields()["phi"].astype(np.float64)
    g = torch.from_numpy((2 * (phiT - target)).astype(np.float32)).to(dev)
    scratch = torch.empty(pf.pflbm_adjoint_scratch_bytes(d.h, T, every), dtype=torch.uint8,
                          device=dev)
    dphi0 = torch.empty_like(phi0_t)
    d.synchronize()
    ds, dm = pf.pflbm_adjoint_run(d.h, phi0_t, T, every, g, dphi0, scratch)
    return ds, dm, dphi0.cpu().numpy().astype(np.float64), phiT


def _oracle_J(orc, nx, ny, wall, p, phi0, target, T):
    s = orc.Sim(nx, ny, wall, orc.Params(**p), phi0.astype(np.float64)).step(T)
    return float(np.sum((s.h.sum(0) - target) ** 2))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("wall", [False, True])
def test_adjoint_matches_fp64_finite_differences(pf, orc, form, wall):
    nx, ny, phi0, target, p = _case(wall, form)
    T, every = 12, 5  # three segments, the last one short
    ds, dm, dphi0, _ = _gpu_adjoint(pf, nx, ny, wall, p, phi0, target, T, every)
    e = 1e-6
    J = lambda **kw: _oracle_J(orc, nx, ny, wall, {**p, **kw}, phi0, target, T)
    fd_s = (J(sigma=p["sigma"] * (1 + e)) - J(sigma=p["sigma"] * (1 - e))) / (2 * e * p["sigma"])
    fd_m = (J(M=p["M"] * (1 + e)) - J(M=p["M"] * (1 - e))) / (2 * e * p["M"])
    v = np.random.default_rng(1).standard_normal(phi0.shape)
    Jp = _oracle_J(orc, nx, ny, wall, p, phi0.astype(np.float64) + e * v, target, T)
    Jm = _oracle_J(orc, nx, ny, wall, p, phi0.astype(np.float64) - e * v, target, T)
    fd_v = (Jp - Jm) / (2 * e)
    ad_v = float(np.sum(dphi0 * v))
    for name, a, b in (("sigma", ds, fd_s), ("M", dm, fd_m), ("phi0.v", ad_v, fd_v)):
        assert abs(a - b) <= 1e-4 * abs(b) + 1e-7, (name, a, b)


@pytest.mark.parametrize("form", ["STF1", "CSF1"])
def test_adjoint_matches_float32_forward_differences(pf, form):
    """Central differences of the CUDA forward itself.  Float32 rounding
    moves J of this case by ~4e-6 between runs with perturbed parameters, so
    the step is 1e-2 relative (J differences ~1e-3, truncation O(1e-4)) and
    the bound 1e-2; the 1e-4 bar is met against the FP64 oracle above."""
    import torch
    wall = True
    nx, ny, phi0, target, p = _case(wall, form)
    T = 12
    ds, dm, _, _ = _gpu_adjoint(pf, nx, ny, wall, p, phi0, target, T, 4)

    def J(**kw):
        d = pf.Domain(nx, ny, wall_y=wall).set_params(**{**p, **kw}).init_phi(phi0)
        d.step(T)
        return float(np.sum((d.fields()["phi"].astype(np.float64) - target) ** 2))
    e = 1e-2
    fd_s = (J(sigma=p["sigma"] * (1 + e)) - J(sigma=p["sigma"] * (1 - e))) / (2 * e * p["sigma"])
    fd_m = (J(M=p["M"] * (1 + e)) - J(M=p["M"] * (1 - e))) / (2 * e * p["M"])
    assert abs(ds - fd_s) <= 1e-2 * abs(fd_s), (ds, fd_s)
    assert abs(dm - fd_m) <= 1e-2 * abs(fd_m), (dm, fd_m)


def test_checkpoint_interval_does_not_change_gradients(pf):
    nx, ny, phi0, target, p = _case(True, "CSF1")
    T = 12
    res = [_gpu_adjoint(pf, nx, ny, True, p, phi0, target, T, k) for k in (1, 5, 12)]
    for ds, dm, dphi0, _ in res[1:]:
        assert abs(ds - res[0][0]) <= 1e-6 * abs(res[0][0])
        assert abs(dm - res[0][1]) <= 1e-6 * abs(res[0][1])
        assert np.abs(dphi0 - res[0][2]).max() <= 1e-6 * np.abs(res[0][2]).max()


def test_autograd_function(pf):
    import torch
    from paper_2012_14729_gb300 import adjoint
    nx, ny, phi0, target, p = _case(False, "STF2")
    T = 10
    dev = torch.device("cuda")
    spec = adjoint.RunSpec(nx, ny, False, T, 4, {k: v for k, v in p.items()
                                                  if k not in ("sigma", "M")})
    phi0_t = torch.from_numpy(phi0).to(dev).requires_grad_(True)
    sigma = torch.tensor(p["sigma"], dtype=torch.float64, requires_grad=True)
    M = torch.tensor(p["M"], dtype=torch.float64, requires_grad=True)
    phiT = adjoint.run(phi0_t, sigma, M, spec)
    J = ((phiT.double() - torch.from_numpy(target).to(dev).double()) ** 2).sum()
    J.backward()
    ds, dm, dphi0, _ = _gpu_adjoint(pf, nx, ny, False, p, phi0, target, T, 4)
    assert abs(sigma.grad.item() - ds) <= 1e-5 * abs(ds)
    assert abs(M.grad.item() - dm) <= 1e-5 * abs(dm)
    assert np.abs(phi0_t.grad.cpu().numpy() - dphi0).max() <= 1e-5 * np.abs(dphi0).max()


def test_domain_left_at_final_state(pf):
    import torch
    nx, ny, phi0, target, p = _case(True, "PF2")
    T = 9
    ref = pf.Domain(nx, ny, wall_y=True).set_params(**p).init_phi(phi0)
    ref.step(T)
    d = pf.Domain(nx, ny, wall_y=True).set_params(**p)
    dev = torch.device("cuda")
    phi0_t = torch.from_numpy(phi0).to(dev)
    g = torch.zeros_like(phi0_t)
    scratch = torch.empty(pf.pflbm_adjoint_scratch_bytes(d.h, T, 4), dtype=torch.uint8, device=dev)
    pf.pflbm_adjoint_run(d.h, phi0_t, T, 4, g, torch.empty_like(phi0_t), scratch)
    assert d.t == T
    for a, b in zip(d.populations(), ref.populations()):
        np.testing.assert_array_equal(a, b)


def test_legacy_stream_runs_without_graphs(pf):
    """On the legacy default stream (which cannot be captured) the segments
    run as plain launches: the gradients equal those of a graph replay."""
    import torch
    nx, ny, phi0, target, p = _case(True, "STF2")
    T, every = 10, 4
    out = []
    for stream in (None, torch.cuda.default_stream()):
        d = pf.Domain(nx, ny, wall_y=True, stream=stream).set_params(**p)
        dev = torch.device("cuda")
        phi0_t = torch.from_numpy(phi0).to(dev)
        g = torch.from_numpy(target).to(dev)
        scratch = torch.empty(pf.pflbm_adjoint_scratch_bytes(d.h, T, every), dtype=torch.uint8,
                              device=dev)
        dphi0 = torch.empty_like(phi0_t)
        torch.cuda.synchronize()
        ds, dm = pf.pflbm_adjoint_run(d.h, phi0_t, T, every, g, dphi0, scratch)
        out.append((ds, dm, dphi0.cpu().numpy()))
    # parameter gradients are FP64 atomic sums (order may vary): 1e-12
    assert abs(out[0][0] - out[1][0]) <= 1e-12 * abs(out[0][0])
    assert abs(out[0][1] - out[1][1]) <= 1e-12 * abs(out[0][1])
    np.testing.assert_array_equal(out[0][2], out[1][2])


def test_adjoint_on_a_larger_walled_grid(pf, orc):
    """640 x 420 nodes (268 800, ragged in y for the reverse tail's 32 x 8
    tiles), moving walls, gravity and a density contrast: the reverse sweep
    on a grid of many tiles against central differences of the FP64
    oracle."""
    import torch
    nx, ny, wall, form = 640, 420, True, "CSF1"
    phi0 = wl.drop(nx, ny, 60.0, 4.0, xc=301.7, yc=209.6, periodic_y=False).astype(np.float32)
    target = wl.drop(nx, ny, 64.0, 4.0, periodic_y=False).astype(np.float32)
    p = dict(sigma=0.02, W=4.0, M=0.1, rho1=1.0, rho2=0.5, nu1=0.1, nu2=0.05, gy=-1e-5,
             uw_bottom=-0.01, uw_top=0.01, form=form)
    p["rho0"] = float(np.mean(0.5 * (1 + phi0) + 0.25 * (1 - phi0)))
    T, every = 8, 3
    ds, dm, _, _ = _gpu_adjoint(pf, nx, ny, wall, p, phi0, target, T, every)
    e = 1e-6
    J = lambda **kw: _oracle_J(orc, nx, ny, wall, {**p, **kw}, phi0, target, T)
    fd_s = (J(sigma=p["sigma"] * (1 + e)) - J(sigma=p["sigma"] * (1 - e))) / (2 * e * p["sigma"])
    fd_m = (J(M=p["M"] * (1 + e)) - J(M=p["M"] * (1 - e))) / (2 * e * p["M"])
    assert abs(ds - fd_s) <= 1e-4 * abs(fd_s) + 1e-7, (ds, fd_s)
    assert abs(dm - fd_m) <= 1e-4 * abs(fd_m) + 1e-7, (dm, fd_m)
