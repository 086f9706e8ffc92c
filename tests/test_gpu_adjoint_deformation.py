"""GPU test of the adjoint on the deformation objective of Sec. 5.5: the
gradient of the Taylor deformation J = D(phi_T) = (L - B)/(L + B) with
respect to sigma, M and the initial phi, against central differences of the
FP64 oracle (D of the oracle's phi_T, oracle.taylor_D).

The case keeps D well away from 0, where it is well conditioned: an initially
elliptic drop (semi-axes R(1 +- 0.15), D_0 ~ 0.15) between walls moving at
-/+0.02 on a 96 x 64 lattice, 240 steps checkpointed every 80.  dD/dphi_T is
the exact derivative of D written with torch (float64 autograd of the same
moment formula, on the host); the adjoint carries it back through the
discrete float32 scheme."""
import math

import numpy as np
import pytest

from paper_2012_14729_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

NX, NY, T, EVERY = 96, 64, 240, 80


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_14729_gb300 import build, pflbm
    build.build()
    pflbm.load()
    return pflbm


def _case(form):
    phi0 = wl.ellipse(NX, NY, 16.0, 4.0, e=0.15, xc=47.6, yc=31.7)
    p = dict(sigma=4e-3, W=4.0, M=0.05, rho1=1.0, rho2=1.0, nu1=0.1, nu2=0.1,
             uw_bottom=-0.02, uw_top=0.02, form=form, rho0=1.0)
    return phi0.astype(np.float32), p


def _D_and_grad(phi):
    """Taylor D of phi (second moments of w = (1 + phi)/2 about its centroid,
    L, B = 4 sqrt of the eigenvalues) and dD/dphi, float64 autograd."""
    import torch
    t = torch.tensor(phi, dtype=torch.float64, requires_grad=True)
    w = 0.5 * (1 + t)
    ny, nx = phi.shape
    y = torch.arange(ny, dtype=torch.float64)[:, None]
    x = torch.arange(nx, dtype=torch.float64)[None, :]
    m = w.sum()
    cx, cy = (w * x).sum() / m, (w * y).sum() / m
    sxx = (w * (x - cx) ** 2).sum() / m
    syy = (w * (y - cy) ** 2).sum() / m
    sxy = (w * (x - cx) * (y - cy)).sum() / m
    tr, det = sxx + syy, sxx * syy - sxy * sxy
    disc = torch.sqrt(tr * tr / 4 - det)
    L, B = 4 * torch.sqrt(tr / 2 + disc), 4 * torch.sqrt(tr / 2 - disc)
    D = (L - B) / (L + B)
    D.backward()
    return float(D.detach()), t.grad.numpy()


def _oracle_D(orc, p, phi0):
    s = orc.Sim(NX, NY, True, orc.Params(**p), phi0.astype(np.float64)).step(T)
    return orc.taylor_D(s.macro())


@pytest.mark.parametrize("form", ["STF1", "CSF1"])
def test_taylor_deformation_gradient_matches_fp64_differences(pf, orc, form):
    import torch
    phi0, p = _case(form)
    dev = torch.device("cuda")
    d = pf.Domain(NX, NY, wall_y=True).set_params(**p)
    phi0_t = torch.from_numpy(phi0).to(dev)
    d.init_phi(phi0_t)
    d.step(T)
    DT, g = _D_and_grad(d.fields()["phi"].astype(np.float64))
    assert DT > 0.05, DT  # away from the ill-conditioned D ~ 0
    gt = torch.from_numpy(g.astype(np.float32)).to(dev)
    scratch = torch.empty(pf.pflbm_adjoint_scratch_bytes(d.h, T, EVERY), dtype=torch.uint8,
                          device=dev)
    dphi0 = torch.empty_like(phi0_t)
    d.synchronize()
    ds, dm = pf.pflbm_adjoint_run(d.h, phi0_t, T, EVERY, gt, dphi0, scratch)
    dphi0 = dphi0.cpu().numpy().astype(np.float64)

    e = 1e-6
    J = lambda **kw: _oracle_D(orc, {**p, **kw}, phi0)
    fd_s = (J(sigma=p["sigma"] * (1 + e)) - J(sigma=p["sigma"] * (1 - e))) / (2 * e * p["sigma"])
    fd_m = (J(M=p["M"] * (1 + e)) - J(M=p["M"] * (1 - e))) / (2 * e * p["M"])
    # a direction that moves the interface: a bump in the normal direction
    Y, X = np.mgrid[0:NY, 0:NX].astype(float)
    v = np.exp(-((X - 66.0) ** 2 + (Y - 34.0) ** 2) / 40.0) * (1 - phi0.astype(np.float64) ** 2)
    Jp = _oracle_D(orc, p, phi0.astype(np.float64) + e * v)
    Jm = _oracle_D(orc, p, phi0.astype(np.float64) - e * v)
    fd_v = (Jp - Jm) / (2 * e)
    ad_v = float(np.sum(dphi0 * v))
    print(f"TAYLOR-D {form}: D_T = {DT:.4f}; dD/dsigma {ds:.6e} vs {fd_s:.6e}; dD/dM {dm:.6e} "
          f"vs {fd_m:.6e}; dD/dphi0.v {ad_v:.6e} vs {fd_v:.6e}")
    for name, a, b in (("sigma", ds, fd_s), ("M", dm, fd_m), ("phi0.v", ad_v, fd_v)):
        assert math.isfinite(a) and abs(a - b) <= 1e-4 * abs(b), (name, a, b, abs(a - b) / abs(b))
