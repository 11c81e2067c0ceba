"""Pins of the oracle's Monte Carlo collisions, secondary emission, births and
external circuit.

* Null-collision MCC ([14] via Section 3): a mono-energetic electron population
  collides in one step as a binomial sample with probability
  (1 - exp(-nu_max dt)) nu_k(E) / nu_max for process k; the counts are checked
  at 4.5 sigma.  Energy bookkeeping is exact: excitation removes 11.55 eV,
  ionization 15.76 eV (Section 3, reactions 1b, 1c), elastic loses
  2 m/M (1 - cos chi) of E with chi the actual deflection angle.
* Secondary emission (Section 3): yield gamma per ion impact on the cathode,
  electron born at the impact point with zero velocity; the impact charge drives
  the external circuit V_c = -V_s + I R_ext (Sections 3 and 6).
* Table 1 rows 1-4 satisfy the circuit relation within the table's rounding.
* Births get ids next_id, next_id + 1, ... in order of (parent id, kind).
"""
import math
import os

import numpy as np
import pytest

import oracle
import pic_inputs
from pic_inputs import E_CHARGE, M_ELECTRON, M_ARGON, K_BOLTZMANN


def _empty():
    return {k: np.zeros(0) for k in ("r", "z", "vr", "vt", "vz")} | {"id": np.zeros(0, np.int64)}


def _mcc_params(**kw):
    p = pic_inputs.params_rz32()
    p.update(push_on=0, field_on=0, b_mode=1, B0r=0.0, B0z=0.0, gamma_i=0.0, gamma_e=0.0,
             mcc_on=1, weight=1.0)
    p.update(kw)
    return p


def _mono_electrons(n, E_eV, p, seed=3):
    rng = np.random.default_rng(seed)
    v = math.sqrt(2 * E_eV * E_CHARGE / M_ELECTRON)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    r = p["R"] * np.sqrt(rng.random(n)) * 0.99
    z = p["L"] * (0.05 + 0.9 * rng.random(n))
    return {"r": r, "z": z, "vr": v * d[0], "vt": v * d[1], "vz": v * d[2],
            "id": np.arange(n, dtype=np.int64)}


def test_cross_section_stand_ins_closed_forms():
    p = pic_inputs.params_rz32()
    s = oracle.sigma(p, 100.0)
    assert s[0] == 1e-19
    assert s[2] == pytest.approx(2.8e-20, rel=0.02)
    # excitation peaks at E = e * E_ex (maximum of ln(x)/x) with C/(e E_ex^2)
    Epk = math.e * p["exc_E"]
    assert oracle.sigma(p, Epk)[1] == pytest.approx(p["exc_C"] / (math.e * p["exc_E"] ** 2), rel=1e-12)
    assert oracle.sigma(p, Epk * 1.01)[1] < oracle.sigma(p, Epk)[1]
    assert oracle.sigma(p, Epk * 0.99)[1] < oracle.sigma(p, Epk)[1]
    assert oracle.sigma(p, 11.0)[1] == 0.0 and oracle.sigma(p, 15.0)[2] == 0.0


def test_nu_max_bounds_every_energy():
    p = pic_inputs.params_rz32()
    numax = oracle.nu_max(p)
    Es = np.concatenate([np.geomspace(1e-3, p["E_cap"], 3000), [p["E_cap"]]])
    nus = []
    for E in Es:
        s = oracle.sigma(p, E)
        nus.append(p["n_gas"] * s.sum() * math.sqrt(2 * E * E_CHARGE / M_ELECTRON))
    nus = np.array(nus)
    assert (nus <= numax).all()
    assert numax <= 1.0011 * nus.max()


@pytest.mark.parametrize("E0", [100.0, 30.0])
def test_collision_counts_binomial(E0):
    p = _mcc_params()
    n = 400000
    parts = {"e": _mono_electrons(n, E0, p), "i": _empty()}
    orc = oracle.Oracle(p, parts, solve=False)
    orc.step(1)
    d = orc.diag()
    numax = oracle.nu_max(p)
    pnull = -math.expm1(-numax * p["dt"])
    s = oracle.sigma(p, E0)
    v = math.sqrt(2 * E0 * E_CHARGE / M_ELECTRON)
    for k, key in enumerate(("n_elastic", "n_excite", "n_ionize")):
        prob = pnull * p["n_gas"] * s[k] * v / numax
        mean, sd = n * prob, math.sqrt(n * prob * (1 - prob))
        assert abs(d[key] - mean) <= 4.5 * sd + 1, (key, d[key], mean, sd)
    # total real collisions vs nu_T dt to first order in nu_max dt
    tot = d["n_elastic"] + d["n_excite"] + d["n_ionize"]
    nuT = p["n_gas"] * s.sum() * v
    assert tot / n == pytest.approx(nuT * p["dt"], rel=0.05 + 4.5 / math.sqrt(max(tot, 1)))


def test_collision_energy_bookkeeping():
    E0 = 100.0
    p = _mcc_params()
    n = 300000
    e0 = _mono_electrons(n, E0, p, seed=11)
    orc = oracle.Oracle(p, {"e": e0, "i": _empty()}, solve=False)
    orc.step(1)
    d = orc.diag()
    e1 = orc.get_particles(0)
    ions = orc.get_particles(1)
    old = e1["id"] < n
    idx = e1["id"][old]
    v_old = np.stack([e0["vr"][idx], e0["vt"][idx], e0["vz"][idx]])
    v_new = np.stack([e1["vr"][old], e1["vt"][old], e1["vz"][old]])
    E_new = 0.5 * M_ELECTRON * (v_new ** 2).sum(0) / E_CHARGE
    changed = np.abs(E_new - E0) > 1e-9 * E0
    moved = np.abs(v_new - v_old).max(0) > 1e-9 * np.abs(v_old).max()
    # excitation: exactly E0 - 11.55 eV
    exc = np.abs(E_new - (E0 - p["exc_E"])) < 1e-9 * E0
    assert exc.sum() == d["n_excite"]
    # ionization primaries: E <= E0 - I
    ionp = E_new <= E0 - p["ion_I"] + 1e-9
    assert ionp.sum() == d["n_ionize"]
    # elastic: E'/E = 1 - 2 m/M (1 - cos chi), chi the actual deflection
    el = moved & ~exc & ~ionp
    assert el.sum() == d["n_elastic"]
    cosc = (v_old[:, el] * v_new[:, el]).sum(0) / (
        np.linalg.norm(v_old[:, el], axis=0) * np.linalg.norm(v_new[:, el], axis=0))
    np.testing.assert_allclose(E_new[el] / E0, 1 - 2 * M_ELECTRON / p["m_ion"] * (1 - cosc),
                               rtol=1e-12)
    # isotropic: mean cos chi ~ 0
    assert abs(cosc.mean()) < 4.5 / math.sqrt(3 * el.sum())
    # ionization: secondaries and ions born in pairs, energies add to E0 - I
    new_e = ~old
    assert new_e.sum() == d["n_ionize"] == ions["id"].shape[0]
    E_sec = 0.5 * M_ELECTRON * (e1["vr"][new_e] ** 2 + e1["vt"][new_e] ** 2 + e1["vz"][new_e] ** 2) / E_CHARGE
    assert E_new[ionp].sum() + E_sec.sum() == pytest.approx(d["n_ionize"] * (E0 - p["ion_I"]), rel=1e-12)
    # ions born thermal at the gas temperature
    vi = np.stack([ions["vr"], ions["vt"], ions["vz"]])
    sig2 = K_BOLTZMANN * p["T_gas"] / M_ARGON
    nion = vi.shape[1]
    assert abs(vi.mean()) < 5 * math.sqrt(sig2 / (3 * nion))
    assert (vi ** 2).mean() == pytest.approx(sig2, rel=5 * math.sqrt(2 / (3 * nion)))
    assert not changed[~moved].any()


def _ion_beam(p, hits_per_step, nsteps, r_hit, speed=2.0e4):
    """Ions placed so that `hits_per_step[k]` of them cross z = 0 during step k."""
    dt = p["dt"]
    rs, zs, ids = [], [], []
    nid = 0
    for k in range(nsteps):
        for j in range(hits_per_step[k]):
            rs.append(r_hit)
            zs.append((k + 0.5) * speed * dt)
            ids.append(nid)
            nid += 1
    n = len(rs)
    return {"r": np.array(rs), "z": np.array(zs), "vr": np.zeros(n), "vt": np.zeros(n),
            "vz": np.full(n, -speed), "id": np.array(ids, dtype=np.int64)}


def _circuit_params(**kw):
    p = pic_inputs.params_rz32()
    p.update(field_on=0, b_mode=1, B0r=0.0, B0z=0.0, mcc_on=0, gamma_i=0.0, gamma_e=0.0,
             circuit_mode=1, Vs=300.0, Rext=3000.0, n_avg=4)
    p.update(kw)
    return p


@pytest.mark.parametrize("gamma", [0.0, 1.0])
def test_circuit_prescribed_cathode_charge(gamma):
    hits = [3, 0, 5, 2, 7, 1, 0, 4]
    p = _circuit_params(gamma_i=gamma, weight=1.0e6)
    ions = _ion_beam(p, hits, len(hits), r_hit=0.01)
    orc = oracle.Oracle(p, {"e": _empty(), "i": ions})
    fac = 1.0 + gamma      # each impact also emits one electron when gamma = 1
    for k in range(len(hits)):
        orc.step(1)
        d = orc.diag()
        lo = max(0, k - p["n_avg"] + 1)
        q = [fac * E_CHARGE * p["weight"] * h for h in hits[lo:k + 1]]
        I = sum(q) / (len(q) * p["dt"])
        V = min(0.0, max(-p["Vs"], -p["Vs"] + I * p["Rext"]))
        assert d["I_cath"] == pytest.approx(I, rel=1e-13)
        assert d["V_cath"] == pytest.approx(V, rel=1e-13, abs=1e-12)
        assert d["n_ion_cath"] == hits[k]
        assert d["n_sey"] == (hits[k] if gamma == 1.0 else 0)


def test_circuit_clamps_to_ground():
    p = _circuit_params(Rext=1.0e9, weight=1.0e6)
    orc = oracle.Oracle(p, {"e": _empty(), "i": _ion_beam(p, [5], 1, 0.01)})
    orc.step(1)
    assert orc.diag()["V_cath"] == 0.0


def test_ions_outside_cathode_radius_do_not_count():
    p = _circuit_params(weight=1.0e6, gamma_i=1.0)
    orc = oracle.Oracle(p, {"e": _empty(), "i": _ion_beam(p, [4], 1, r_hit=0.021)})
    orc.step(1)
    d = orc.diag()
    assert d["n_ion_cath"] == 0 and d["I_cath"] == 0.0 and d["V_cath"] == -p["Vs"]


def test_table1_rows_obey_the_circuit(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "table1_circuit.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, sey, R, I, V, ok = line.split()
                rows.append((name, float(sey), float(R), float(I), float(V), int(ok)))
    assert len(rows) == 11
    steps = 4
    for name, sey, R, I_mA, V_mag, ok in rows:
        # drive the oracle's circuit with a constant cathode current of I_mA
        per_step = 10
        p = _circuit_params(Vs=300.0, Rext=R, n_avg=steps, gamma_i=0.0)
        p["weight"] = I_mA * 1e-3 * p["dt"] / (per_step * E_CHARGE)
        orc = oracle.Oracle(p, {"e": _empty(), "i": _ion_beam(p, [per_step] * steps, steps, 0.01)})
        orc.step(steps)
        V = orc.diag()["V_cath"]
        assert V == pytest.approx(-300.0 + I_mA * 1e-3 * R, rel=1e-12)
        if ok:
            assert abs(abs(V) - V_mag) <= 10.0, name
        else:
            assert abs(abs(V) - V_mag) > 10.0, name


def test_birth_ids_follow_parent_order():
    # ions hitting the cathode with gamma = 1: each emits an electron at its
    # impact radius; ids go out in the order of the parent ion ids
    p = _circuit_params(gamma_i=1.0, weight=1.0, circuit_mode=0, Vc_fixed=0.0)
    n = 6
    rng = np.random.default_rng(5)
    r_hits = rng.random(n) * 0.015
    ions = {"r": r_hits, "z": np.full(n, 0.5 * 2e4 * p["dt"]), "vr": np.zeros(n),
            "vt": np.zeros(n), "vz": np.full(n, -2e4),
            "id": np.array([40, 12, 33, 7, 25, 18], dtype=np.int64)}
    electrons = _mono_electrons(3, 1.0, p)
    electrons["id"] = np.array([100, 101, 102], dtype=np.int64)
    orc = oracle.Oracle(p, {"e": electrons, "i": ions})
    next_id = orc.next_id
    assert next_id == 103
    orc.step(1)
    e = orc.get_particles(0)
    born = e["id"] >= next_id
    order = np.argsort(ions["id"])
    np.testing.assert_array_equal(np.sort(e["id"][born]), np.arange(next_id, next_id + n))
    by_id = np.argsort(e["id"][born])
    np.testing.assert_allclose(e["r"][born][by_id], r_hits[order], rtol=1e-15)
    assert (e["z"][born] == 0.0).all() and (e["vr"][born] == 0.0).all()


# ---- reaction (1d): stepwise ionization from the metastable Ar* (Section 3) ----
def test_metastable_cross_section_closed_forms():
    p = pic_inputs.params_rz32()
    I = p["meta_I"]
    assert I == 4.20 and oracle.sigma_meta(p, 4.19) == 0.0 and oracle.sigma_meta(p, I) == 0.0
    # Lotz form a ln(E/I)/(E I): maximum at E = e I with value a / (e I^2)
    Epk = math.e * I
    assert oracle.sigma_meta(p, Epk) == pytest.approx(p["meta_a"] / (math.e * I * I), rel=1e-12)
    assert oracle.sigma_meta(p, Epk * 1.01) < oracle.sigma_meta(p, Epk)
    assert oracle.sigma_meta(p, 100.0) == pytest.approx(
        p["meta_a"] * math.log(100.0 / I) / (100.0 * I), rel=1e-12)


def test_nu_max_bounds_every_energy_with_metastables():
    p = pic_inputs.params_rz32()
    p["n_meta"] = 2.5e17
    numax = oracle.nu_max(p)
    Es = np.concatenate([np.geomspace(1e-3, p["E_cap"], 3000), [p["E_cap"]]])
    nus = np.array([(p["n_gas"] * oracle.sigma(p, E).sum() + p["n_meta"] * oracle.sigma_meta(p, E))
                    * math.sqrt(2 * E * E_CHARGE / M_ELECTRON) for E in Es])
    assert (nus <= numax).all()
    assert numax <= 1.0011 * nus.max()
    p0 = dict(p, n_meta=0.0)
    assert numax > oracle.nu_max(p0)


def test_metastable_ionization_counts_binomial():
    # only the metastable process: no ground-state gas, a dense Ar* background
    E0 = 30.0
    p = _mcc_params(n_gas=0.0, n_meta=3e20)
    n = 300000
    parts = {"e": _mono_electrons(n, E0, p, seed=5), "i": _empty()}
    orc = oracle.Oracle(p, parts, solve=False)
    orc.step(1)
    d = orc.diag()
    assert d["n_elastic"] == d["n_excite"] == d["n_ionize"] == 0
    numax = oracle.nu_max(p)
    pnull = -math.expm1(-numax * p["dt"])
    v = math.sqrt(2 * E0 * E_CHARGE / M_ELECTRON)
    prob = pnull * p["n_meta"] * oracle.sigma_meta(p, E0) * v / numax
    mean, sd = n * prob, math.sqrt(n * prob * (1 - prob))
    assert d["n_ionize_meta"] > 100
    assert abs(d["n_ionize_meta"] - mean) <= 4.5 * sd + 1, (d["n_ionize_meta"], mean, sd)


def test_metastable_ionization_energy_bookkeeping():
    E0 = 30.0
    p = _mcc_params(n_gas=0.0, n_meta=3e20)
    n = 200000
    e0 = _mono_electrons(n, E0, p, seed=7)
    orc = oracle.Oracle(p, {"e": e0, "i": _empty()}, solve=False)
    orc.step(1)
    d = orc.diag()
    e1, ions = orc.get_particles(0), orc.get_particles(1)
    old = e1["id"] < n
    E_new = 0.5 * M_ELECTRON * (e1["vr"][old] ** 2 + e1["vt"][old] ** 2 + e1["vz"][old] ** 2) / E_CHARGE
    prim = E_new <= E0 - p["meta_I"] + 1e-9
    assert prim.sum() == d["n_ionize_meta"] == (~old).sum() == ions["id"].shape[0]
    E_sec = 0.5 * M_ELECTRON * (e1["vr"][~old] ** 2 + e1["vt"][~old] ** 2 + e1["vz"][~old] ** 2) / E_CHARGE
    # each event removes exactly the 4.20 eV threshold
    assert E_new[prim].sum() + E_sec.sum() == pytest.approx(
        d["n_ionize_meta"] * (E0 - p["meta_I"]), rel=1e-12)
    # electrons that did not collide keep E0
    assert np.abs(E_new[~prim] - E0).max() < 1e-9 * E0
