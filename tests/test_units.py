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
