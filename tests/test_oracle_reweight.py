"""Pins of the oracle's particle re-weighting and particles-per-cell count.

Section 6 (large-grid EC/MC runs): once the particles per cell pass ~1000, two
thirds of the particles are removed and the weight of the others tripled.
The oracle keeps each particle independently with probability 1/factor by a
counter-based draw of its id, so:

* the kept count is binomial(n, 1/factor): checked at 5 sigma;
* kept records are unchanged, in their old order, and the kept set does not
  depend on the storage order;
* weight x factor: total charge, the density profile (chi-square over radial
  and axial bins) and the mean kinetic energy are conserved in expectation;
* factor 1 is the identity; factor < 1 is refused.

The particles-per-cell maximum is checked against a brute-force histogram of
the particle positions.
"""
import math

import numpy as np
import pytest

import oracle
import pic_inputs
from pic_inputs import E_CHARGE, M_ELECTRON


def _plasma(n=30000, seed=4, **kw):
    p = pic_inputs.params_rz32(seed=seed)
    p.update(kw)
    p, parts = pic_inputs.seed_plasma(p, n, n0=1e15, seed=seed + 1)
    return p, parts


def _oracle(p, parts):
    return oracle.Oracle(p, parts, solve=False)


def test_kept_fraction_binomial_and_weight():
    p, parts = _plasma()
    o = _oracle(p, parts)
    n = parts["e"]["r"].size
    kept = o.reweight(3)
    ne, ni = o.count(0), o.count(1)
    assert kept == ne + ni
    sd = math.sqrt(n * (1 / 3) * (2 / 3))
    for k in (ne, ni):
        assert abs(k - n / 3) < 5 * sd, (k, n / 3)
    assert o.weight == pytest.approx(3.0 * p["weight"], rel=0, abs=0)
    # the two species draw independently (keyed by species): same ids -> different sets
    e_ids = set(o.get_particles(0)["id"].tolist())
    i_ids = set((o.get_particles(1)["id"] - n).tolist())
    both = len(e_ids & i_ids)
    assert abs(both - n / 9) < 5 * math.sqrt(n * (1 / 9) * (8 / 9)), both


def test_kept_records_unchanged_and_order_independent():
    p, parts = _plasma(n=5000)
    o = _oracle(p, parts)
    o.reweight(3)
    ke = o.get_particles(0)
    src = parts["e"]
    pos = np.searchsorted(src["id"], ke["id"])
    assert np.all(np.diff(pos) > 0)          # old order kept
    for f in ("r", "z", "vr", "vt", "vz"):
        assert np.array_equal(ke[f], src[f][pos])
    # reversed storage order: the same set
    rev = {k: v[::-1].copy() for k, v in src.items()}
    o2 = oracle.Oracle(p, {"e": rev, "i": parts["i"]}, solve=False)
    o2.reweight(3)
    assert set(o2.get_particles(0)["id"].tolist()) == set(ke["id"].tolist())
    # a later step index draws a different, independent set
    o3 = _oracle(p, parts)
    o3.set_circuit(0.0, 7)
    o3.reweight(3)
    ids3 = set(o3.get_particles(0)["id"].tolist())
    common = len(ids3 & set(ke["id"].tolist()))
    n = src["r"].size
    assert abs(common - n / 9) < 5 * math.sqrt(n / 9 * 8 / 9)


def test_charge_profile_and_energy_conserved_in_expectation():
    p, parts = _plasma(n=60000)
    n = parts["e"]["r"].size
    o = _oracle(p, parts)
    o.reweight(3)
    ke = o.get_particles(0)
    w = o.weight
    # total represented electrons: 3 * kept vs n (binomial, 5 sigma)
    assert abs(w * ke["r"].size - p["weight"] * n) < 5 * p["weight"] * 3 * math.sqrt(n * 2 / 9)
    # density profile: counts in 8 radial x 8 axial bins against n/3 of the original
    H0, er, ez = np.histogram2d(parts["e"]["r"], parts["e"]["z"], bins=8,
                                range=[[0, p["R"]], [0, p["L"]]])
    H1, _, _ = np.histogram2d(ke["r"], ke["z"], bins=[er, ez])
    # each bin: binomial(H0, 1/3); chi-square over 64 bins, 99.99 % bound ~ 120
    chi2 = float(np.sum((H1 - H0 / 3) ** 2 / (H0 * (1 / 3) * (2 / 3))))
    assert chi2 < 120.0, chi2
    # mean kinetic energy of the kept electrons (sampling error of a mean)
    e0 = 0.5 * M_ELECTRON * (parts["e"]["vr"] ** 2 + parts["e"]["vt"] ** 2 + parts["e"]["vz"] ** 2)
    e1 = 0.5 * M_ELECTRON * (ke["vr"] ** 2 + ke["vt"] ** 2 + ke["vz"] ** 2)
    assert abs(e1.mean() - e0.mean()) < 5 * e0.std() / math.sqrt(e1.size) * math.sqrt(2 / 3) * 1.5


def test_factor_one_identity_and_bad_factor():
    p, parts = _plasma(n=2000)
    o = _oracle(p, parts)
    assert o.reweight(1) == 4000
    assert o.weight == p["weight"]
    assert np.array_equal(o.get_particles(1)["id"], parts["i"]["id"])
    with pytest.raises(ValueError):
        o.reweight(0)


def test_new_weight_enters_the_deposit():
    p, parts = _plasma(n=3000)
    # electrons only: the node charges sum to -e w N_e
    empty = {k: v[:0] for k, v in parts["i"].items()}
    o = oracle.Oracle(p, {"e": parts["e"], "i": empty}, solve=False)
    o.reweight(3)
    o.solve_fields()
    Q = o.fields()["Q"]
    assert Q.sum() == pytest.approx(-E_CHARGE * 3 * p["weight"] * o.count(0), rel=1e-12)


def test_ppc_max_is_the_histogram_maximum():
    p, parts = _plasma(n=20000)
    p.update(mcc_on=1)
    o = oracle.Oracle(p, parts)
    o.step(3)
    d = o.diag()
    for sp, key in ((0, "ppc_max_e"), (1, "ppc_max_i")):
        q = o.get_particles(sp)
        # cell index by the same floor rule as the deposit (last cell closed)
        m = np.minimum(np.floor(q["r"] / (p["R"] / p["nr"])).astype(int), p["nr"] - 1)
        n = np.minimum(np.floor(q["z"] / (p["L"] / p["nz"])).astype(int), p["nz"] - 1)
        h = np.bincount(m * p["nz"] + n, minlength=p["nr"] * p["nz"])
        assert d[key] == h.max(), (key, d[key], h.max())
