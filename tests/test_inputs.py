"""Checks of the seeded synthetic inputs (not of the method): the seed plasma is
uniform in volume and Maxwellian; the grown state has its ring where asked."""
import math

import numpy as np
import pytest

import pic_inputs
from pic_inputs import E_CHARGE, M_ELECTRON


def test_seed_plasma_moments_and_radial_cdf():
    p = pic_inputs.params_rz32()
    p2, parts = pic_inputs.seed_plasma(p, 65536, n0=1e15, seed=0)
    assert p2["weight"] == pytest.approx(1e15 * math.pi * p["R"] ** 2 * p["L"] / 65536)
    e = parts["e"]
    n = e["r"].shape[0]
    sig2 = 2.0 * E_CHARGE / M_ELECTRON
    for k in ("vr", "vt", "vz"):
        assert abs(e[k].mean()) < 4 * math.sqrt(sig2 / n)
        assert e[k].var() == pytest.approx(sig2, rel=4 * math.sqrt(2.0 / n))
    # uniform in volume: r^2/R^2 and z/L are U(0,1); KS distance small
    for u in (np.sort(e["r"] ** 2 / p["R"] ** 2), np.sort(e["z"] / p["L"])):
        ks = np.abs(u - (np.arange(n) + 0.5) / n).max()
        assert ks < 1.63 / math.sqrt(n)  # 1% critical value
    assert (parts["i"]["r"] == e["r"]).all()
    assert set(e["id"]) .isdisjoint(set(parts["i"]["id"]))


def test_grown_ring_state_shape():
    p = pic_inputs.params_rz256()
    p2, parts = pic_inputs.grown_ring_state(p, 200000, seed=2)
    r, z = parts["e"]["r"], parts["e"]["z"]
    assert (r >= 0).all() and (r < p["R"]).all() and (z >= 0).all() and (z < p["L"]).all()
    # density near the ring centre is several times the floor
    V = lambda r0, r1, z0, z1: math.pi * (r1 ** 2 - r0 ** 2) * (z1 - z0)
    ring = ((r > 0.0115) & (r < 0.0135) & (z > 0.0015) & (z < 0.0025)).sum() / V(0.0115, 0.0135, 0.0015, 0.0025)
    floor = ((r > 0.03) & (r < 0.045) & (z > 0.02) & (z < 0.045)).sum() / V(0.03, 0.045, 0.02, 0.045)
    assert 6.0 < ring / floor < 14.0


def test_paper_chamber_preset():
    """Section 3's chamber: 3 x 3 cm, cathode to 0.85 L_r, the rest of z = 0
    insulating, 10 mTorr (n = p / k T), V_ext -300 V; the field stand-in's
    racetrack (B_z = 0) lies between the inner (6.5 mm) and outer (1.7 cm)
    magnets."""
    import oracle
    p = pic_inputs.params_paper()
    assert p["R"] == p["L"] == 0.03 and p["Rc"] == pytest.approx(0.0255)
    assert p["gap_neumann"] == 1 and p["wall_neumann"] == 0
    assert p["n_gas"] == pytest.approx(10e-3 * 133.322368421 / (1.380649e-23 * 300.0))
    assert p["Vs"] == 300.0 and p["gamma_e"] == 0.1
    rs = np.linspace(0.0065, 0.017, 2001)
    bz = np.array([oracle.bfield(p, r, 0.0)[1] for r in rs])
    r0 = rs[np.argmin(np.abs(bz))]
    assert 0.0065 < r0 < 0.017 and abs(r0 - 0.012) < 1e-4
