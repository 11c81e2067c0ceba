"""Pins of the oracle's grid pieces: magnetron field, node volumes, deposit,
Poisson solve and the two field gathers of Section 2.

Facts used (none re-derived from the oracle's own formulas):
* the stand-in field is a vacuum field: div B = 0 and curl B = 0;
  B_z(0, 0) = k A0; B_r vanishes at the first zero of J1 (k r = 3.8317);
* node control volumes tile the cylinder: their sum is pi R^2 L;
* tent weights form a partition of unity and reproduce r (linear) or r^2
  (volume weighting) exactly; a single particle splits in closed form;
* the finite-volume RZ operator is exact on a r^2 + b z^2 + c; smooth
  solutions converge at second order; Gauss's law holds discretely;
* MC-PIC has no axial self-force (symmetry / translation invariance);
* EC-PIC's force is minus the gradient of the field energy (Section 2: E is
  minus sum phi grad S with the deposit's S).
"""
import math

import numpy as np
import pytest

import oracle
import pic_inputs
from pic_inputs import EPS0, E_CHARGE

J1_ZERO = 3.8317059702075125


def small_params(**kw):
    p = pic_inputs.params_rz32()
    p.update(nr=16, nz=24, R=0.02, L=0.03, Rc=0.015)
    p.update(kw)
    return p


def test_bfield_is_divergence_and_curl_free():
    p = pic_inputs.params_rz32()
    h = 1e-6
    k = p["B_k"]
    for r, z in [(0.004, 0.001), (0.011, 0.006), (0.019, 0.02), (0.0235, 0.012)]:
        brp, _ = oracle.bfield(p, r + h, z)
        brm, _ = oracle.bfield(p, r - h, z)
        _, bzp = oracle.bfield(p, r, z + h)
        _, bzm = oracle.bfield(p, r, z - h)
        br0, bz0 = oracle.bfield(p, r, z)
        div = ((r + h) * brp - (r - h) * brm) / (2 * h * r) + (bzp - bzm) / (2 * h)
        brzp, _ = oracle.bfield(p, r, z + h)
        brzm, _ = oracle.bfield(p, r, z - h)
        _, bzrp = oracle.bfield(p, r + h, z)
        _, bzrm = oracle.bfield(p, r - h, z)
        curl = (brzp - brzm) / (2 * h) - (bzrp - bzrm) / (2 * h)
        scale = k * math.hypot(br0, bz0)
        assert abs(div) < 1e-6 * scale
        assert abs(curl) < 1e-6 * scale


def test_bfield_special_values():
    p = pic_inputs.params_rz32()
    br, bz = oracle.bfield(p, 0.0, 0.0)
    assert br == 0.0 and bz == pytest.approx(p["B_kA0"], rel=1e-15)
    br, bz = oracle.bfield(p, J1_ZERO / p["B_k"], 0.0)
    assert abs(br) < 1e-12
    # k r at the cathode edge is 3.83: B_r is three orders below peak there
    br, _ = oracle.bfield(p, 0.02, 0.0)
    assert abs(br) < 1e-3 * p["B_kA0"]
    # decays as exp(-k z) along the axis
    _, bz1 = oracle.bfield(p, 0.0, 0.01)
    assert bz1 == pytest.approx(p["B_kA0"] * math.exp(-p["B_k"] * 0.01), rel=1e-14)


def test_node_volumes_tile_the_cylinder():
    for kw in ({}, {"nr": 7, "nz": 5, "R": 0.013, "L": 0.041}):
        p = small_params(**kw)
        V = oracle.node_volume(p)
        assert V.sum() == pytest.approx(math.pi * p["R"] ** 2 * p["L"], rel=1e-13)
        assert (V > 0).all()


def test_deposit_total_charge_and_moments():
    rng = np.random.default_rng(1)
    for rw in (0, 1):
        p = small_params(rweight=rw)
        n = 20000
        r = p["R"] * np.sqrt(rng.random(n)) * 0.999999
        z = p["L"] * rng.random(n)
        Q = oracle.deposit(p, r, z, 1.0)
        assert Q.sum() == pytest.approx(n, rel=1e-13)
        dr = p["R"] / p["nr"]
        rm = np.arange(p["nr"] + 1) * dr
        # per-particle moments: deposit one particle at a time
        for k in range(50):
            q1 = oracle.deposit(p, r[k:k + 1], z[k:k + 1], 1.0)
            wr = q1.sum(axis=1)
            if rw == 0:
                assert (wr * rm).sum() == pytest.approx(r[k], rel=1e-13)
            else:
                assert (wr * rm ** 2).sum() == pytest.approx(r[k] ** 2, rel=1e-12)
            assert q1.sum() == pytest.approx(1.0, rel=1e-14)


def test_single_particle_split_closed_form():
    p = small_params()
    dr, dz = p["R"] / p["nr"], p["L"] / p["nz"]
    m, n = 3, 5
    Q = oracle.deposit(p, [(m + 0.25) * dr], [(n + 0.5) * dz], 2.0)
    assert Q[m, n] == pytest.approx(2 * 0.75 * 0.5)
    assert Q[m + 1, n] == pytest.approx(2 * 0.25 * 0.5)
    assert Q[m, n + 1] == pytest.approx(2 * 0.75 * 0.5)
    assert Q[m + 1, n + 1] == pytest.approx(2 * 0.25 * 0.5)
    assert np.count_nonzero(Q) == 4
    # volume weighting: S_{m+1} = ((m+1/4)^2 - m^2) / (2m + 1)
    pv = small_params(rweight=1)
    Qv = oracle.deposit(pv, [(m + 0.25) * dr], [(n + 0.5) * dz], 1.0)
    s1 = ((m + 0.25) ** 2 - m ** 2) / (2 * m + 1)
    assert Qv[m + 1, n] == pytest.approx(s1 * 0.5, rel=1e-13)
    assert Qv[m, n] == pytest.approx((1 - s1) * 0.5, rel=1e-13)


def _bc_from(p, f):
    nr, nz = p["nr"], p["nz"]
    dr, dz = p["R"] / nr, p["L"] / nz
    rr = (np.arange(nr + 1) * dr)[:, None]
    zz = (np.arange(nz + 1) * dz)[None, :]
    return f(rr, zz) * np.ones((nr + 1, nz + 1)), rr, zz


def test_poisson_exact_on_quadratics():
    p = small_params()
    a, b, c = 3.0e4, -1.7e4, 12.0
    phi_exact, rr, zz = _bc_from(p, lambda r, z: a * r * r + b * z * z + c)
    rho = np.full(phi_exact.shape, -EPS0 * (4 * a + 2 * b))
    phi = oracle.poisson(p, rho, phi_exact)
    assert np.abs(phi - phi_exact).max() < 1e-11 * np.abs(phi_exact).max()


def test_poisson_second_order_convergence():
    errs = []
    for nr in (16, 32, 64):
        p = small_params(nr=nr, nz=nr, R=0.02, L=0.03)
        R, L = p["R"], p["L"]
        ka, kz = math.pi / (2 * R), math.pi / L

        def phi_f(r, z):
            return np.cos(ka * r) * np.sin(kz * z)

        phi_ex, rr, zz = _bc_from(p, phi_f)
        with np.errstate(invalid="ignore", divide="ignore"):
            sinc = np.where(rr > 0, np.sin(ka * rr) / np.where(rr > 0, rr, 1.0), ka)
        lap = (-ka * ka * np.cos(ka * rr) - ka * sinc - kz * kz * np.cos(ka * rr)) * np.sin(kz * zz)
        rho = -EPS0 * lap
        phi = oracle.poisson(p, rho, np.zeros_like(phi_ex))
        errs.append(np.abs(phi - phi_ex).max())
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    for q in ratios:
        assert 3.7 < q < 4.3, (errs, ratios)


def test_poisson_gauss_law():
    """Total charge equals the outward flux eps0 E . dA through the Dirichlet
    boundary, with the control-volume faces 2 pi r_{m+1/2} dz (radial) and the
    annulus areas (axial) of the finite-volume cells."""
    p = small_params()
    rng = np.random.default_rng(4)
    nr, nz = p["nr"], p["nz"]
    dr, dz = p["R"] / nr, p["L"] / nz
    V = oracle.node_volume(p)
    rho = rng.normal(size=(nr + 1, nz + 1)) * 1e-6
    bc = np.zeros_like(rho)
    bc[: int(p["Rc"] / dr) + 1, 0] = -300.0
    phi = oracle.poisson(p, rho, bc)
    free = np.zeros_like(rho, dtype=bool)
    free[:nr, 1:nz] = True
    charge = (rho * V)[free].sum()
    area = np.array([math.pi * dr * dr / 4] + [2 * math.pi * m * dr * dr for m in range(1, nr + 1)])
    flux = 0.0
    for m in range(nr):
        for n in range(1, nz):
            if n == 1:
                flux += EPS0 * area[m] * (phi[m, 1] - phi[m, 0]) / dz
            if n == nz - 1:
                flux += EPS0 * area[m] * (phi[m, nz - 1] - phi[m, nz]) / dz
            if m == nr - 1:
                flux += EPS0 * 2 * math.pi * (m + 0.5) * dr * dz * (phi[m, n] - phi[nr, n]) / dr
    assert flux == pytest.approx(charge, rel=1e-9, abs=1e-9 * np.abs(rho * V).sum())


def _self_field(p, r, z):
    Q = oracle.deposit(p, [r], [z], E_CHARGE)
    V = oracle.node_volume(p)
    phi = oracle.poisson(p, Q / V, np.zeros_like(Q))
    return oracle.efield_at(p, phi, r, z), phi


@pytest.mark.parametrize("rw", [0, 1])
def test_mc_no_axial_self_force_on_symmetry_plane(rw):
    p = small_params(gather=1, rweight=rw, nz=24)
    L = p["L"]
    for r in (0.0013, 0.0071, 0.0152):
        (er, ez), _ = _self_field(p, r, L / 2)
        assert abs(ez) < 1e-12 * abs(er) + 1e-18


@pytest.mark.parametrize("rw", [0, 1])
def test_mc_no_axial_self_force_translation_invariant(rw):
    # a long cylinder: away from the ends the Green's function is translation
    # invariant in z to exp(-2.405 d / R); MC's self-force then vanishes at any z
    p = small_params(gather=1, rweight=rw, nr=8, nz=240, R=0.008, L=0.24)
    dz = p["L"] / p["nz"]
    ec = dict(p, gather=0)
    for r, z in ((0.0021, 120.3 * dz), (0.0057, 117.81 * dz)):
        (er, ez), phi = _self_field(p, r, z)
        assert abs(ez) < 1e-8 * abs(er)
        # EC does have a self-force in z inside the cell: the pin distinguishes them
        ez_ec = oracle.efield_at(ec, phi, r, z)[1]
        assert abs(ez_ec) > 1e-3 * abs(er)


@pytest.mark.parametrize("rw", [0, 1])
def test_ec_force_is_minus_energy_gradient(rw):
    p = small_params(gather=0, rweight=rw)
    dr, dz = p["R"] / p["nr"], p["L"] / p["nz"]
    V = oracle.node_volume(p)
    rng = np.random.default_rng(7)
    # a fixed background of charges plus the test particle
    rb = p["R"] * np.sqrt(rng.random(40))
    zb = p["L"] * (0.1 + 0.8 * rng.random(40))
    qb = rng.choice([-1.0, 1.0], 40) * E_CHARGE

    def energy(r, z):
        Q = oracle.deposit(p, [r], [z], E_CHARGE)
        for k in range(40):
            Q += oracle.deposit(p, rb[k:k + 1], zb[k:k + 1], qb[k])
        phi = oracle.poisson(p, Q / V, np.zeros_like(Q))
        return 0.5 * (Q * phi).sum(), phi

    for r, z in ((5.37 * dr, 7.61 * dz), (0.42 * dr, 11.2 * dz), (12.9 * dr, 3.3 * dz)):
        W0, phi = energy(r, z)
        er, ez = oracle.efield_at(p, phi, r, z)
        h_r, h_z = 1e-4 * dr, 1e-4 * dz
        fr = -(energy(r + h_r, z)[0] - energy(r - h_r, z)[0]) / (2 * h_r)
        fz = -(energy(r, z + h_z)[0] - energy(r, z - h_z)[0]) / (2 * h_z)
        scale = abs(E_CHARGE) * math.hypot(er, ez)
        assert abs(E_CHARGE * er - fr) < 1e-6 * scale
        assert abs(E_CHARGE * ez - fz) < 1e-6 * scale
        # with grounded walls 1/2 Q.phi equals the edge-sum field energy
        assert oracle.field_energy(p, phi) == pytest.approx(W0, rel=1e-10)
