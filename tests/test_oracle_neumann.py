"""Pins of the oracle's insulating (Neumann) boundaries (Section 3: the block
beside the cathode that is not part of it is a Neumann boundary, letting the
potential float between cathode and anode).

Facts used:
* the finite-volume operator is exact for potentials quadratic in r and in z
  whose normal derivative vanishes on the insulating parts, when each node
  carries the exact charge of its control volume: phi = a (r^2 - 2 R r) +
  b z^2 + c has d phi/dz = 0 on z = 0 and d phi/dr = 0 on r = R, and
  rho = -eps0 (4a + 2b - 2 a R / r) integrates in closed form over annuli;
* an insulating plane z = 0 is a mirror: the solution equals that of the
  domain doubled to [-L, L] with the charge and the boundary values mirrored
  and conductors only (the same oracle, all-Dirichlet path);
* the MC-PIC nodal field has no normal component on an insulating wall.
"""
import math

import numpy as np
import pytest

import oracle
import pic_inputs
from pic_inputs import EPS0


def small_params(**kw):
    p = pic_inputs.params_rz32()
    p.update(nr=16, nz=24, R=0.02, L=0.03, Rc=0.012)
    p.update(kw)
    return p


def _grid(p):
    nr, nz = p["nr"], p["nz"]
    dr, dz = p["R"] / nr, p["L"] / nz
    return nr, nz, dr, dz


def _exact_charge_density(p, a, b):
    """rho per node such that rho * V = the exact charge of the node's control
    volume for rho(r) = -eps0 (4a + 2b - 2 a R / r)."""
    nr, nz, dr, dz = _grid(p)
    R = p["R"]
    V = oracle.node_volume(p)
    rho = np.empty((nr + 1, nz + 1))
    for m in range(nr + 1):
        r1, r2 = max(0.0, (m - 0.5) * dr), min(R, (m + 0.5) * dr)
        radial = (4 * a + 2 * b) * (r2 * r2 - r1 * r1) / 2 - 2 * a * R * (r2 - r1)
        for n in range(nz + 1):
            z1, z2 = max(0.0, (n - 0.5) * dz), min(p["L"], (n + 0.5) * dz)
            q = -EPS0 * 2 * math.pi * (z2 - z1) * radial
            rho[m, n] = q / V[m, n]
    return rho


@pytest.mark.parametrize("gap,wall", [(1, 1), (1, 0), (0, 1)])
def test_exact_on_quadratics_with_insulating_walls(gap, wall):
    p = small_params(gap_neumann=gap, wall_neumann=wall)
    nr, nz, dr, dz = _grid(p)
    a, b, c = 3.0e4, -1.7e4, 12.0
    R = p["R"]
    rr = (np.arange(nr + 1) * dr)[:, None]
    zz = (np.arange(nz + 1) * dz)[None, :]
    # zero normal derivative on every insulating part; the conducting parts
    # take their Dirichlet values from the same function
    ar = a * (rr * rr - 2 * R * rr) if wall else a * rr * rr
    phi_ex = ar + b * zz * zz + c + 0 * rr * zz
    rho = _exact_charge_density(p, a, b) if wall else np.full(phi_ex.shape, -EPS0 * (4 * a + 2 * b))
    phi = oracle.poisson(p, rho, phi_ex)
    assert np.abs(phi - phi_ex).max() < 1e-11 * np.abs(phi_ex).max()
    # the insulating nodes are unknowns (a conductor there would hold the
    # given value whatever the charge): perturbing the charge moves them
    phi2 = oracle.poisson(p, rho * 1.01, phi_ex)
    m_gap = int(p["Rc"] / dr) + 2
    moved = abs(phi2[m_gap, 0] - phi[m_gap, 0]) > 0 if gap else phi2[m_gap, 0] == phi[m_gap, 0]
    assert moved
    assert (abs(phi2[nr, nz // 2] - phi[nr, nz // 2]) > 0) == bool(wall)


def test_insulating_plane_is_a_mirror():
    nr, nz = 12, 10
    p = small_params(nr=nr, nz=nz, R=0.015, L=0.0125, Rc=-1.0, gap_neumann=1)
    rng = np.random.default_rng(9)
    rho = rng.normal(size=(nr + 1, nz + 1)) * 1e-6
    bc = np.zeros((nr + 1, nz + 1))
    bc[:, nz] = rng.normal(size=nr + 1) * 10.0      # anode values
    bc[nr, :] = rng.normal(size=nz + 1) * 10.0      # conducting wall values
    phi = oracle.poisson(p, rho, bc)
    # doubled domain [0, 2L], its row nz is the insulating plane
    p2 = small_params(nr=nr, nz=2 * nz, R=0.015, L=0.025, Rc=-1.0, gap_neumann=0)
    rho2 = np.concatenate([rho[:, :0:-1], rho], axis=1)
    bc2 = np.concatenate([bc[:, :0:-1], bc], axis=1)
    phi2 = oracle.poisson(p2, rho2, bc2)
    assert np.abs(phi2[:, nz:] - phi).max() <= 1e-12 * np.abs(phi).max()
    assert np.abs(phi2[:, nz::-1] - phi).max() <= 1e-12 * np.abs(phi).max()


def test_mc_nodal_field_has_no_normal_component_on_insulators():
    rng = np.random.default_rng(2)
    for gap, wall in ((1, 1), (0, 0)):
        p = small_params(gather=1, gap_neumann=gap, wall_neumann=wall)
        nr, nz, dr, dz = _grid(p)
        phi = rng.normal(size=(nr + 1, nz + 1))
        r_gap = p["Rc"] + 2.5 * dr                 # between two gap nodes
        _, ez = oracle.efield_at(p, phi, r_gap, 0.0)
        er, _ = oracle.efield_at(p, phi, p["R"] * (1 - 1e-13), 0.4 * p["L"])
        if gap:
            assert ez == 0.0 and abs(er) < 1e-9
        else:
            assert ez != 0.0 and abs(er) > 1e-3
        # on the cathode the normal field stays
        _, ez_c = oracle.efield_at(p, phi, 0.3 * p["Rc"], 0.0)
        assert ez_c != 0.0
