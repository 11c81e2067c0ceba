"""Pins of the oracle's step diagnostics against closed forms.

* Peak density (Section 4's density profiles): the largest number density of
  a species over the nodes after the step, a node's density being its
  deposited charge over its control volume.  Hand-built states put all of a
  species' macroparticles exactly on chosen nodes (push and collisions off,
  so they stay there).  The expected control volume is computed here from
  the geometry alone -- the part of the cylinder within half a cell of the
  node, pi (r_hi^2 - r_lo^2) (z_hi - z_lo) clipped at the axis and the walls
  -- not from the oracle's own volume formula: the axis node's disk of radius
  dr/2, the half volume of a node on z = 0, both at the corner.
* Kinetic energy time-centring: K = sum 1/2 m w (|v^{n-1/2}|^2 + |v^{n+1/2}|^2) / 2.
  In a uniform axial field E0 with no magnetic field, one step changes v_z by
  exactly q E0 dt / m, so K is known in closed form; taking K from either
  half-step velocity alone misses it by far more than the tolerance.
* Field energy of that uniform field: 1/2 eps0 E0^2 pi R^2 L, the energy of a
  uniform field filling the cylinder.
"""
import math

import numpy as np
import pytest

import oracle
import pic_inputs
from pic_inputs import E_CHARGE, EPS0, M_ELECTRON


def _params():
    p = pic_inputs.params_rz32()
    p.update(nr=8, nz=8, R=0.008, L=0.008, Rc=0.004, mcc_on=0, push_on=0, circuit_mode=0,
             Vc_fixed=0.0, b_mode=1, B0r=0.0, B0z=0.0, weight=1e6)
    return p


def _control_volume(p, m, n):
    dr, dz = p["R"] / p["nr"], p["L"] / p["nz"]
    r_lo, r_hi = max(0.0, (m - 0.5) * dr), min(p["R"], (m + 0.5) * dr)
    z_lo, z_hi = max(0.0, (n - 0.5) * dz), min(p["L"], (n + 0.5) * dz)
    return math.pi * (r_hi ** 2 - r_lo ** 2) * (z_hi - z_lo)


def _on_nodes(p, counts, id0=0):
    """counts: {(m, n): k} -> k particles at rest on node (m, n) (on the outer
    wall m = nr: a relative 1e-13 inside it, the domain being r < R)."""
    dr, dz = p["R"] / p["nr"], p["L"] / p["nz"]
    r, z = [], []
    for (m, n), k in counts.items():
        r += [m * dr if m < p["nr"] else p["R"] * (1.0 - 1e-13)] * k
        z += [n * dz] * k
    k = len(r)
    v = np.zeros(k)
    return dict(r=np.array(r), z=np.array(z), vr=v, vt=v.copy(), vz=v.copy(),
                id=np.arange(id0, id0 + k, dtype=np.int64))


# (electrons, ions, the node where each species' density peaks); in the first
# two the peak is not at the node holding the most particles
CASES = [
    ({(0, 4): 3, (5, 5): 40}, {(3, 0): 7, (6, 3): 12}, (0, 4), (3, 0)),   # axis; z = 0
    ({(0, 0): 2, (4, 4): 30}, {(0, 7): 5, (2, 6): 9}, (0, 0), (0, 7)),    # corner; axis
    ({(6, 6): 12, (1, 2): 1}, {(8, 4): 12, (7, 7): 20}, (6, 6), (8, 4)),  # interior; r = R
]


@pytest.mark.parametrize("electrons, ions, peak_e, peak_i", CASES)
def test_peak_density_of_hand_built_states(electrons, ions, peak_e, peak_i):
    p = _params()
    parts = {"e": _on_nodes(p, electrons), "i": _on_nodes(p, ions, id0=1000)}
    orc = oracle.Oracle(p, parts)
    orc.step(1)
    d = orc.diag()
    for key, counts, node in (("n_e_peak", electrons, peak_e), ("n_i_peak", ions, peak_i)):
        dens = {nd: k * p["weight"] / _control_volume(p, *nd) for nd, k in counts.items()}
        assert max(dens, key=dens.get) == node
        assert d[key] == pytest.approx(dens[node], rel=1e-10), (key, dens)


def test_kinetic_energy_is_centred_on_the_step():
    p = _params()
    p.update(push_on=1)
    dz = p["L"] / p["nz"]
    E0 = -2.5e4                       # V/m along z: phi = -E0 z
    v_old = np.array([3.0e5, -2.0e5, 1.0e5])
    e = dict(r=np.array([0.0041]), z=np.array([0.0043]), vr=v_old[:1], vt=v_old[1:2],
             vz=v_old[2:], id=np.array([0], dtype=np.int64))
    i = dict(r=np.array([0.0052]), z=np.array([0.0031]), vr=np.array([1.0e3]),
             vt=np.array([0.0]), vz=np.array([-2.0e3]), id=np.array([1], dtype=np.int64))
    orc = oracle.Oracle(p, {"e": e, "i": i})
    z_nodes = np.arange(p["nz"] + 1) * dz
    phi = np.tile(-E0 * z_nodes, (p["nr"] + 1, 1))
    orc.set_phi(phi)
    orc.step(1)
    d = orc.diag()
    w = p["weight"]
    checks = [("K_e", M_ELECTRON, -E_CHARGE, v_old),
              ("K_i", p["m_ion"], E_CHARGE, np.array([1.0e3, 0.0, -2.0e3]))]
    for key, mass, q, v in checks:
        dv = q * E0 * p["dt"] / mass
        v2_old = float(v @ v)
        v2_new = v2_old - v[2] ** 2 + (v[2] + dv) ** 2
        K = 0.5 * mass * w * 0.5 * (v2_old + v2_new)
        assert d[key] == pytest.approx(K, rel=1e-12), key
        # either half-step velocity alone is far off
        for wrong in (0.5 * mass * w * v2_old, 0.5 * mass * w * v2_new):
            assert abs(wrong - K) > 1e-6 * K
    W = 0.5 * EPS0 * E0 ** 2 * math.pi * p["R"] ** 2 * p["L"]
    assert d["W_field"] == pytest.approx(W, rel=1e-12)
