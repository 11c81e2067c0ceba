"""Pins of the oracle's random numbers and particle push against independent facts.

* Philox4x64-10 against numpy's independent implementation (numpy advances its
  128-bit counter by one before each block, so numpy's first block with
  counter c is Philox(c + 1)).
* Philox4x32-10 (the null-collision candidate draw) against the known-answer
  vectors published with the generator (Salmon et al., SC'11, Random123
  distribution): all-zero, all-ones and the digits of pi as counter and key.
* Boris push closed forms (the paper says only "explicit"; the Boris scheme is
  the reading): in a uniform B the velocity turns by exactly 2 atan(w dt / 2)
  per step and the positions lie on a circle of radius
  r_L sqrt(1 + (w dt / 2)^2); the E x B drift velocity is a fixed point; |v|
  is conserved when E = 0.
"""
import math

import numpy as np
import pytest

import oracle
from pic_inputs import E_CHARGE, M_ELECTRON, M_ARGON


def _numpy_philox(ctr, key, nblocks=1):
    c = np.array(ctr, dtype=np.uint64).copy()
    # numpy's generator increments before producing: feed counter - 1 (with borrow)
    words = [int(x) for x in c]
    val = sum(w << (64 * i) for i, w in enumerate(words))
    val = (val - 1) % (1 << 256)
    c = np.array([(val >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)
    g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=c)
    return g.random_raw(4 * nblocks)


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([1, 0, 0, 0], [0, 0]),
    ([123456789, 42, 2, 0], [7, 1]),
    ([2**64 - 1, 5, 0, 0], [2**63 + 11, 0]),
    ([987, 2**40 + 3, 4, 0], [0xDEADBEEF, 1]),
])
def test_philox_matches_numpy(ctr, key):
    got = oracle.philox4x64(ctr, key)
    ref = _numpy_philox(ctr, key)
    assert [int(x) for x in got] == [int(x) for x in ref]


def test_philox_consecutive_counters_match_numpy_stream():
    key = [3, 1]
    ref = _numpy_philox([10, 0, 0, 0], key, nblocks=5)
    got = np.concatenate([oracle.philox4x64([10 + k, 0, 0, 0], key) for k in range(5)])
    assert [int(x) for x in got] == [int(x) for x in ref]


@pytest.mark.parametrize("ctr,key,expected", [
    ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
    ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
    ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
])
def test_philox4x32_known_answers(ctr, key, expected):
    assert [int(x) for x in oracle.philox4x32(ctr, key)] == expected


def _lab_track(q_over_m, dt, E, B, state, nsteps):
    """Run the RZ push and rebuild the lab-frame (x, y) and velocity vectors."""
    theta = 0.0
    xs, vs = [], []
    s = np.array(state, dtype=float)
    for _ in range(nsteps):
        r_old = s[0]
        s_new = oracle.boris_move(q_over_m, dt, E[0], E[1], B[0], B[1], s)
        # The frame angle advance: the particle moved from (r_old, 0) to a point at
        # distance r_new; recover the Cartesian end point from v_theta/v_r rotation.
        # x' = r_old + vx dt, y' = vy dt, with (vx, vy) = R(-dphi) (vr', vt').
        vr, vt = s_new[2], s_new[3]
        # the frame rotation dphi satisfies r_new cos(dphi) = r_old + vx dt,
        # r_new sin(dphi) = vy dt; with (vx, vy) = (vr cos - vt sin, vr sin + vt cos)
        # -> solve by iterating the fixed point (converges in a few rounds).
        dphi = 0.0
        for _ in range(60):
            c, sn = math.cos(dphi), math.sin(dphi)
            vx, vy = vr * c - vt * sn, vr * sn + vt * c
            dphi = math.atan2(vy * dt, r_old + vx * dt)
        theta += dphi
        c, sn = math.cos(theta), math.sin(theta)
        xs.append((s_new[0] * c, s_new[0] * sn, s_new[1]))
        vs.append((vr * c - vt * sn, vr * sn + vt * c, s_new[4]))
        s = s_new
    return np.array(xs), np.array(vs)


def test_larmor_rotation_angle_and_radius():
    B = 0.02
    q_over_m = -E_CHARGE / M_ELECTRON
    omega = abs(q_over_m) * B
    dt = 0.3 / omega                      # omega dt = 0.3
    v_perp = 1.0e6
    r_l = v_perp / omega
    # start 5 Larmor radii off axis, moving in theta
    state = [5 * r_l, 0.0, 0.0, v_perp, 0.0]
    xs, vs = _lab_track(q_over_m, dt, (0.0, 0.0), (0.0, B), state, 400)
    # velocity turns by exactly 2 atan(omega dt / 2) per step
    ang = np.arctan2(vs[1:, 1], vs[1:, 0]) - np.arctan2(vs[:-1, 1], vs[:-1, 0])
    ang = (ang + np.pi) % (2 * np.pi) - np.pi
    np.testing.assert_allclose(np.abs(ang), 2 * math.atan(omega * dt / 2), rtol=1e-9)
    # positions on a circle of radius r_L sqrt(1 + (omega dt/2)^2)
    p = xs[:, :2]
    a, b, c = p[0], p[1], p[2]
    d = 2 * (a[0] * (b[1] - c[1]) + b[0] * (c[1] - a[1]) + c[0] * (a[1] - b[1]))
    ux = ((a @ a) * (b[1] - c[1]) + (b @ b) * (c[1] - a[1]) + (c @ c) * (a[1] - b[1])) / d
    uy = ((a @ a) * (c[0] - b[0]) + (b @ b) * (a[0] - c[0]) + (c @ c) * (b[0] - a[0])) / d
    rad = np.hypot(p[:, 0] - ux, p[:, 1] - uy)
    np.testing.assert_allclose(rad, r_l * math.sqrt(1 + (omega * dt / 2) ** 2), rtol=1e-8)
    # speed conserved to round-off
    sp = np.linalg.norm(vs, axis=1)
    np.testing.assert_allclose(sp, v_perp, rtol=1e-12)


def test_exb_drift_is_fixed_point():
    # far from the axis (r = 1 km) the RZ frame is locally Cartesian
    Ez, Br = 1.0e3, 0.01
    vd = Ez / Br                            # E x B = (0,0,Ez) x (Br,0,0) -> +theta
    for q_over_m in (-E_CHARGE / M_ELECTRON, E_CHARGE / M_ARGON):
        state = [1.0e3, 0.0, 0.0, vd, 0.0]
        dt = 1e-11
        s = np.array(state)
        for _ in range(200):
            s = oracle.boris_move(q_over_m, dt, 0.0, Ez, Br, 0.0, s)
        assert abs(s[3] - vd) / vd < 1e-6
        assert abs(s[4]) / vd < 1e-6


def test_exb_drift_average_from_rest():
    # from rest, the orbit gyrates about the drift: the mean theta velocity over
    # whole Boris periods equals E/B
    Ez, Br = 2.0e3, 0.02
    q_over_m = -E_CHARGE / M_ELECTRON
    omega = abs(q_over_m) * Br
    theta_step = 2 * math.atan(0.25)        # choose omega dt = 0.5
    dt = 0.5 / omega
    n_per = 2 * math.pi / theta_step
    nsteps = int(round(20 * n_per))
    # choose dt so that an integer number of steps makes 20 turns exactly
    target = 20 * 2 * math.pi / nsteps
    dt = 2 * math.tan(target / 2) / omega
    s = np.array([1.0e3, 0.0, 0.0, 0.0, 0.0])
    vt_sum = 0.0
    for _ in range(nsteps):
        s = oracle.boris_move(q_over_m, dt, 0.0, Ez, Br, 0.0, s)
        vt_sum += s[3]
    assert abs(vt_sum / nsteps - Ez / Br) / (Ez / Br) < 1e-6


def test_speed_conserved_in_magnetron_field_without_E():
    import pic_inputs
    params = pic_inputs.params_rz32()
    s = np.array([0.012, 0.003, 3e5, -2e6, 1e6])
    v0 = np.linalg.norm(s[2:])
    for _ in range(2000):
        br, bz = oracle.bfield(params, s[0], s[1])
        s = oracle.boris_move(-E_CHARGE / M_ELECTRON, 5e-11, 0.0, 0.0, br, bz, s)
    assert abs(np.linalg.norm(s[2:]) - v0) / v0 < 1e-12
