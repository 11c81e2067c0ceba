"""Pins of the oracle's region diagnostics (Sections 4, 5 and 7).

* Sheath, pre-sheath, bulk: a hand-built state whose cells hold chosen numbers
  of ions and electrons and whose potential is a parabola in z gives sheath
  and bulk edges that follow from the definitions by hand (sheath ends where
  n_e >= n_i / 2, bulk starts where E_z = -d phi/dz turns >= 0).
* Electron temperature by region: each cell holds electrons with velocities
  d +- u along one axis (plus a drift d), whose second-moment temperature is
  m_e u^2 / (3 e) whatever the drift; each region gets its own u.
* Cathode ion energy distribution: ions arriving field-free with known
  energies land in the bins floor(E / width); ions outside the radial band
  and electrons are not counted, energies above the top edge overflow.
"""
import math

import numpy as np
import pytest

import oracle
import pic_inputs
from pic_inputs import E_CHARGE, M_ELECTRON, M_ARGON


def _params(**kw):
    p = pic_inputs.params_rz32()
    p.update(nr=32, nz=24, R=0.02, L=0.012, Rc=0.018, mcc_on=0, push_on=0, gamma_i=0.0,
             band_r_lo=0.010, band_r_hi=0.015)
    p.update(kw)
    return p


def _parts(rows):
    out = {}
    for k in ("e", "i"):
        a = np.array(rows[k], dtype=float).reshape(-1, 5)
        n = a.shape[0]
        base = 0 if k == "e" else 10 ** 6
        out[k] = dict(r=a[:, 0].copy(), z=a[:, 1].copy(), vr=a[:, 2].copy(), vt=a[:, 3].copy(),
                      vz=a[:, 4].copy(), id=np.arange(base, base + n, dtype=np.int64))
    return out


def test_sheath_bulk_edges_and_temperatures():
    p = _params()
    nr, nz = p["nr"], p["nz"]
    dr, dz = p["R"] / nr, p["L"] / nz
    NS, NB = 3, 7                      # expected edges (cell indices)
    u = {0: 2.0e6, 1: 1.0e6, 2: 5.0e5}   # per-region velocity spread (m/s)
    drift = 3.0e5
    band = [m for m in range(nr) if p["band_r_lo"] <= (m + 0.5) * dr <= p["band_r_hi"]]
    rows = {"e": [], "i": []}
    for m in band:
        rc = (m + 0.5) * dr
        for n in range(nz):
            zc = (n + 0.5) * dz
            reg = 0 if n < NS else (1 if n < NB else 2)
            # sheath cells: 2 electrons vs 5 ions (2*2 < 5); later cells: 2 vs 2
            ni = 5 if n < NS else 2
            rows["i"] += [[rc, zc, 0.0, 0.0, 0.0]] * ni
            rows["e"] += [[rc, zc, drift + u[reg], 0.0, 0.0], [rc, zc, drift - u[reg], 0.0, 0.0]]
    o = oracle.Oracle(p, _parts(rows), solve=False)
    zn = np.arange(nz + 1)
    # maximum on node NB: -d phi/dz < 0 in cells below it, > 0 from cell NB on
    phi = np.tile(-10.0 * (zn - NB) ** 2.0, (nr + 1, 1))
    o.set_phi(phi)
    for _ in range(2):
        o.region_sample()
    d = o.regions()
    assert d["samples"] == 2
    assert d["z_sheath"] == pytest.approx(NS * dz, rel=1e-14)
    assert d["z_bulk"] == pytest.approx(NB * dz, rel=1e-14)
    for m in band:
        assert d["zs"][m] == pytest.approx(NS * dz) and d["zb"][m] == pytest.approx(NB * dz)
    assert d["ncell"] == [NS * len(band), (NB - NS) * len(band), (nz - NB) * len(band)]
    for reg in range(3):
        T = M_ELECTRON * u[reg] ** 2 / (3 * E_CHARGE)
        assert d["Te"][reg] == pytest.approx(T, rel=1e-9), reg
    # clearing
    o.region_reset()
    assert o.regions()["samples"] == 0 and o.regions()["ncell"] == [0, 0, 0]


def test_cathode_ion_energy_distribution():
    p = _params(push_on=1, field_on=0, b_mode=1, B0r=0.0, B0z=0.0, ied_bins=100,
                ied_emax=200.0)
    de = p["ied_emax"] / p["ied_bins"]
    groups = [(0.012, 101.0, 7), (0.0125, 37.3, 5), (0.005, 80.0, 4), (0.014, 250.0, 3)]
    rows = {"e": [], "i": []}
    for r, E, cnt in groups:
        vz = -math.sqrt(2 * E * E_CHARGE / M_ARGON)
        z = 0.5 * abs(vz) * p["dt"]           # crosses z = 0 within the step
        rows["i"] += [[r, z, 0.0, 0.0, vz]] * cnt
    # electrons crossing in the band are not part of the ion distribution
    vze = -math.sqrt(2 * 50.0 * E_CHARGE / M_ELECTRON)
    rows["e"] += [[0.012, 0.5 * abs(vze) * p["dt"], 0.0, 0.0, vze]] * 6
    o = oracle.Oracle(p, _parts(rows), solve=False)
    o.step(1)
    assert o.diag()["n_ion_cath"] == 19 and o.diag()["n_e_cath"] == 6
    h, over = o.ied()
    want = np.zeros(p["ied_bins"], dtype=np.int64)
    want[int(101.0 // de)] += 7
    want[int(37.3 // de)] += 5
    assert np.array_equal(h, want)
    assert over == 3                       # 250 eV above the 200 eV top edge
    assert o.regions()["ion_impacts"] == 15  # the 80 eV group hit outside the band
