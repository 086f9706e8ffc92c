"""The dimensionless front-end (Sec. 2.3 groups -> lattice parameters)."""
import math

import pytest

from paper_2012_14729_gb300 import units


def test_round_trip_of_the_groups():
    p = units.lattice_params(Lc=128, Uc=0.01, Re=35, We=125, Cn=4 / 128, Pe=300, Fr=0.8,
                             rho_ratio=10, mu_ratio=10)
    g = units.groups(p, Lc=128, Uc=0.01)
    for k, v in dict(Re=35, We=125, Cn=4 / 128, Pe=300, Fr=0.8, rho_ratio=10,
                     mu_ratio=10).items():
        assert g[k] == pytest.approx(v, rel=1e-12), k


def test_capillary_wave_groups_of_the_paper():
    """Sec. 5.3: rho1 = rho2, nu = 0.01, sigma = 0.25, H = 1, Uc = sqrt(sigma /
    (H rho1)) give Re = 50 and We = 1; in lattice units with H = 80 nodes and
    nu = 0.02 the same groups fix Uc = 0.0125 and sigma = 0.0125."""
    Uc_phys = math.sqrt(0.25 / 1.0 / 1.0)
    assert Uc_phys * 1.0 / 0.01 == pytest.approx(50)
    p = units.lattice_params(Lc=80, Uc=0.0125, Re=50, We=1, Cn=4 / 80)
    assert p["nu1"] == pytest.approx(0.02) and p["nu2"] == pytest.approx(0.02)
    assert p["sigma"] == pytest.approx(0.0125) and p["W"] == pytest.approx(4)
    # default Peclet number 1 / Cn, no gravity
    assert units.groups(p, 80, 0.0125)["Pe"] == pytest.approx(20)
    assert p["gy"] == 0.0


def test_rejects_non_positive_groups():
    with pytest.raises(ValueError):
        units.lattice_params(Lc=64, Uc=0.01, Re=0, We=1, Cn=0.1)


def test_rising_bubble_groups_of_the_paper():
    """Sec. 5.4, Table test_Paras: rho1 = 1000, mu1 = 10, g = 0.98, sigma =
    24.5, R = 0.25 with L = 2R and Ug = sqrt(2 R g) give Re = 35, Eo = 10 and
    Mo = Eo^3 / Re^4; the lattice workload keeps those groups."""
    from paper_2012_14729_gb300 import workloads as wl
    si = dict(rho1=1000.0, rho2=100.0, nu1=10.0 / 1000.0, nu2=1.0 / 100.0, sigma=24.5,
              W=0.01, M=1.0, gx=0.0, gy=-0.98)
    Ug = math.sqrt(2 * 0.25 * 0.98)
    g = units.groups(si, Lc=0.5, Uc=Ug)
    assert g["Re"] == pytest.approx(35.0) and g["Eo"] == pytest.approx(10.0)
    assert g["Mo"] == pytest.approx(10.0 ** 3 / 35.0 ** 4)
    assert g["Fr"] == pytest.approx(1.0) and g["We"] == pytest.approx(g["Eo"])
    assert g["rho_ratio"] == pytest.approx(10.0) and g["mu_ratio"] == pytest.approx(10.0)
    for nx in (120, 240):
        c = wl.rising_bubble("STF1", nx=nx)
        gl = units.groups(c.params, Lc=nx / 2, Uc=math.sqrt(-c.params["gy"] * nx / 2))
        for k in ("Re", "Eo", "Mo", "rho_ratio", "mu_ratio"):
            assert gl[k] == pytest.approx(g[k], rel=1e-12), k
        assert gl["Fr"] == pytest.approx(1.0)
        # one second is 1 / s_per_step steps; U_g in SI is Ug lattice x (m/s per lattice)
        assert c.meta["mps_per_lattice"] * math.sqrt(-c.params["gy"] * nx / 2) == \
            pytest.approx(Ug)
