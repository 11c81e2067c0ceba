"""Helpers of the GPU-vs-oracle parity tests: seeded test states and
per-species comparisons by particle id."""
from __future__ import annotations

import math

import numpy as np
import pytest

import pic_inputs
from pic_inputs import E_CHARGE, M_ELECTRON

PARTICLE_TOL = 1e-12   # ||a - b||_inf / ||b||_inf per species and quantity group (FP64)
FIELD_TOL = 1e-10      # ||phi_a - phi_b||_inf / ||phi_b||_inf (FP64)


def busy_state(p: dict, ppc: int, seed: int, Te_eV: float = 40.0, frac_cathode: float = 0.05):
    """A seeded state in which one step exercises every branch: energetic
    electrons (collisions of all kinds, births), ions and electrons about to
    hit the cathode (tally, secondary emission), particles leaving through
    z = L and r = R."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = p["nr"] * p["nz"] * ppc
    p2, parts = pic_inputs.seed_plasma(p, n, seed=seed, Te_eV=Te_eV)
    dt = p["dt"]
    e, i = parts["e"], parts["i"]
    k = int(frac_cathode * n)
    # ions: just above the cathode, falling in at 2e4 m/s
    i["z"][:k] = rng.random(k) * 2e4 * dt
    i["vz"][:k] = -2e4
    i["r"][:k] = p["R"] * np.sqrt(rng.random(k)) * 0.999
    # electrons: a few falling into the cathode
    e["z"][:k] = rng.random(k) * 1e6 * dt
    e["vz"][:k] = -1e6 - np.abs(e["vz"][:k])
    # some particles at the far walls, moving out
    e["z"][k:2 * k] = p["L"] - rng.random(k) * 1e6 * dt
    e["vz"][k:2 * k] = 1e6 + np.abs(e["vz"][k:2 * k])
    i["r"][k:2 * k] = p["R"] - rng.random(k) * 1e4 * dt
    i["vr"][k:2 * k] = 1e4
    return p2, parts


def sort_by_id(d: dict) -> dict:
    o = np.argsort(d["id"], kind="stable")
    return {k: v[o] for k, v in d.items()}


def compare_species(a: dict, b: dict) -> dict:
    """Relative max-norm errors of positions and velocities of two particle
    sets with identical ids (asserted)."""
    a, b = sort_by_id(a), sort_by_id(b)
    assert a["id"].shape == b["id"].shape, (a["id"].shape, b["id"].shape)
    assert np.array_equal(a["id"], b["id"]), "particle id sets differ"
    if a["id"].shape[0] == 0:
        return {"pos": 0.0, "vel": 0.0}
    pa, pb = np.stack([a["r"], a["z"]]), np.stack([b["r"], b["z"]])
    va, vb = np.stack([a["vr"], a["vt"], a["vz"]]), np.stack([b["vr"], b["vt"], b["vz"]])
    return {"pos": float(np.abs(pa - pb).max() / np.abs(pb).max()),
            "vel": float(np.abs(va - vb).max() / max(np.abs(vb).max(), 1e-300))}


def field_err(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def electron_energy_eV(d: dict) -> np.ndarray:
    return 0.5 * M_ELECTRON * (d["vr"] ** 2 + d["vt"] ** 2 + d["vz"] ** 2) / E_CHARGE


def thermal_speed(T_eV: float, mass: float) -> float:
    return math.sqrt(T_eV * E_CHARGE / mass)


COUNT_KEYS = ("N_e", "N_i", "n_ion_cath", "n_e_cath", "n_sey", "n_ionize", "n_excite",
              "n_elastic", "n_ionize_meta", "ppc_max_e", "ppc_max_i")


def check_step64(pg, h, orc, instance: int = 0, check_phi: bool = True) -> dict:
    """One FP64 step of instance `instance` of handle h against the oracle
    `orc`: integer counters equal; positions and velocities per species within
    PARTICLE_TOL (identical id sets); node charge of each species and in total
    within 1e-12; phi within FIELD_TOL; I, V_c within 1e-12; energies and
    peak densities within 1e-10.  Returns the GPU diagnostics."""
    de, do = pg.pic_diagnostics(h, instance), orc.diag()
    for key in COUNT_KEYS:
        assert de[key] == do[key], (instance, key, de[key], do[key])
    for sp in (0, 1):
        err = compare_species(pg.pic_get_particles(h, instance, sp), orc.get_particles(sp))
        assert err["pos"] <= PARTICLE_TOL and err["vel"] <= PARTICLE_TOL, (instance, sp, err)
        qs = field_err(pg.pic_get_species_charge(h, instance, sp), orc.species_charge(sp))
        assert qs <= 1e-12, (instance, sp, qs)
    fg, fo = pg.pic_get_fields(h, instance), orc.fields()
    assert field_err(fg["Q"], fo["Q"]) <= 1e-12
    if check_phi:
        assert field_err(fg["phi"], fo["phi"]) <= FIELD_TOL
    for key in ("I_cath", "V_cath"):
        assert de[key] == pytest.approx(do[key], rel=1e-12, abs=1e-12), (instance, key)
    for key in ("K_e", "K_i", "W_field", "n_e_peak", "n_i_peak"):
        assert de[key] == pytest.approx(do[key], rel=1e-10), (instance, key)
    return de
