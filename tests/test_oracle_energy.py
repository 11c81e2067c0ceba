"""EC-PIC vs MC-PIC energy behaviour when the Debye length is under-resolved
(Section 5: MC-PIC grid-heats when the cell exceeds lambda_De; EC-PIC does
not have that instability for a stationary plasma).

A 2 eV, 1e15 m^-3 plasma (lambda_De = 0.33 mm) on 0.78 mm cells (2.4
lambda_De), no collisions, no magnetic field, reflecting particle walls and
grounded field walls: the total energy W + K of the MC-PIC run must grow
steadily, that of the EC-PIC run must stay within a small drift, and the
MC-PIC growth must be many times the EC-PIC drift.
"""
import numpy as np

import oracle
import pic_inputs


def _run(gather, steps):
    p = pic_inputs.params_rz32(gather=gather)
    p.update(nr=16, nz=16, R=0.0125, L=0.0125, mcc_on=0, walls_reflect=1, circuit_mode=0,
             Vc_fixed=0.0, b_mode=1, B0r=0.0, B0z=0.0)
    p, parts = pic_inputs.seed_plasma(p, 16 * 16 * 16, n0=1e15, seed=1)
    o = oracle.Oracle(p, parts)
    tot = []
    for _ in range(steps):
        o.step(1)
        d = o.diag()
        tot.append(d["W_field"] + d["K_e"] + d["K_i"])
    tot = np.array(tot)
    return tot / tot[0] - 1.0


def test_mc_grid_heating_vs_ec_bounded():
    steps = 4000
    ec = _run(0, steps)
    mc = _run(1, steps)
    q = steps // 4
    mc_q = [mc[i * q:(i + 1) * q].mean() for i in range(4)]
    assert all(b > a for a, b in zip(mc_q, mc_q[1:])), mc_q
    assert mc[-q:].mean() > 0.05
    assert abs(ec).max() < 0.015
    assert mc[-q:].mean() > 8.0 * abs(ec[-q:].mean())
