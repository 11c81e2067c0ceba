"""GPU parity of the FP32 particle mode against the FP64 oracle.

Bar (FP32 mode): positions and velocities within ||a - b||_inf / ||b||_inf <=
1e-5 per species, phi and Q within 1e-5.  A discrete decision taken in FP32
(a collision process chosen by U nu_max against cumulative frequencies, a wall
crossing, the reference axis of a scattering's azimuth -- the incident
direction's smallest component, where two components nearly tie) can fall on
the other side of a threshold than in FP64; a particle whose velocity misses
the bar is counted as such a flip and excluded from the norms, and at most
ceil(1e-5 N) flips are allowed.
"""
import math

import numpy as np
import pytest

import oracle
import pic_inputs
from parity import busy_state, field_err, sort_by_id

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def pg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_10727_gb300 as pg
    return pg


def compare32(a: dict, b: dict):
    """GPU FP32 particles `a` vs oracle FP64 particles `b` (dicts of arrays)."""
    ia, ib = set(a["id"].tolist()), set(b["id"].tolist())
    flips = len(ia ^ ib)
    common = np.array(sorted(ia & ib), dtype=np.int64)
    a, b = sort_by_id(a), sort_by_id(b)
    sa = np.isin(a["id"], common)
    sb = np.isin(b["id"], common)
    A = {k: v[sa] for k, v in a.items()}
    B = {k: v[sb] for k, v in b.items()}
    va = np.stack([A["vr"], A["vt"], A["vz"]])
    vb = np.stack([B["vr"], B["vt"], B["vz"]])
    vmax = max(np.abs(vb).max(), 1e-300) if vb.size else 1.0
    # a particle whose velocity misses the bar took another discrete decision
    branch = np.abs(va - vb).max(axis=0) > TOL32 * vmax
    flips += int(branch.sum())
    keep = ~branch
    if keep.sum() == 0:
        return {"pos": 0.0, "vel": 0.0}, flips
    pa, pb = np.stack([A["r"], A["z"]])[:, keep], np.stack([B["r"], B["z"]])[:, keep]
    return ({"pos": float(np.abs(pa - pb).max() / np.abs(pb).max()),
             "vel": float(np.abs(va[:, keep] - vb[:, keep]).max() / vmax)}, flips)


def _pair32(pg, p, parts):
    p = pic_inputs.with_capacity(p, parts, factor=2.0)
    orc = oracle.Oracle(p, parts)
    h = pg.pic_create(dict(p, precision=1))
    for k, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, 0, sp, parts[k])
    pg.pic_set_phi(h, 0, orc.fields()["phi"])
    return p, orc, h


def _check(pg, h, orc):
    n_total = 0
    flips_total = 0
    for sp in (0, 1):
        a, b = pg.pic_get_particles(h, 0, sp), orc.get_particles(sp)
        err, flips = compare32(a, b)
        n_total += b["id"].shape[0]
        flips_total += flips
        assert err["pos"] <= TOL32 and err["vel"] <= TOL32, (sp, err)
    assert flips_total <= math.ceil(1e-5 * n_total), flips_total
    fg, fo = pg.pic_get_fields(h, 0), orc.fields()
    assert field_err(fg["Q"], fo["Q"]) <= TOL32
    assert field_err(fg["phi"], fo["phi"]) <= TOL32
    return flips_total


@pytest.mark.parametrize("gather", [0, 1])
@pytest.mark.parametrize("rweight", [0, 1])
def test_fp32_one_step_busy_state(pg, gather, rweight):
    p = pic_inputs.params_rz32(gather=gather)
    p.update(rweight=rweight, gamma_i=0.5, gamma_e=0.3, poisson_tol=1e-12, circuit_mode=1,
             Vs=400.0, Rext=100.0, n_avg=3)
    p, parts = busy_state(p, ppc=16, seed=31 + gather + 2 * rweight)
    p, orc, h = _pair32(pg, p, parts)
    orc.step(1)
    pg.pic_step(h, 1)
    flips = _check(pg, h, orc)
    d, do = pg.pic_diagnostics(h, 0), orc.diag()
    if flips == 0:
        for key in ("N_e", "N_i", "n_ion_cath", "n_e_cath", "n_sey", "n_ionize", "n_excite",
                    "n_elastic"):
            assert d[key] == do[key], key
    assert d["n_ionize"] > 0 and d["n_sey"] > 0


def test_fp32_collision_queue_overflow(pg):
    """A collision-dominated gas (p_null about 0.83): more candidates per chunk
    than the FP32 queue holds (256); the rest run from the per-thread masks."""
    p = pic_inputs.params_rz32()
    p.update(n_gas=200.0 * p["n_gas"], poisson_tol=1e-12, circuit_mode=1, Vs=400.0,
             Rext=100.0, n_avg=3)
    p, parts = busy_state(p, ppc=16, seed=47)
    p, orc, h = _pair32(pg, p, parts)
    orc.step(1)
    pg.pic_step(h, 1)
    _check(pg, h, orc)
    d = pg.pic_diagnostics(h, 0)
    assert d["n_elastic"] + d["n_excite"] + d["n_ionize"] > 2048


def test_fp32_metastable_ionization(pg):
    """Reaction (1d) in FP32 mode against the FP64 oracle (dense Ar* so that
    the step has tens of events)."""
    p = pic_inputs.params_rz32(gather=0)
    p.update(n_meta=3e20, gamma_i=0.2, gamma_e=0.1, poisson_tol=1e-12)
    p, parts = busy_state(p, ppc=16, seed=47)
    p, orc, h = _pair32(pg, p, parts)
    orc.step(1)
    pg.pic_step(h, 1)
    flips = _check(pg, h, orc)
    d, do = pg.pic_diagnostics(h, 0), orc.diag()
    assert do["n_ionize_meta"] > 0
    if flips == 0:
        assert d["n_ionize_meta"] == do["n_ionize_meta"]
    else:
        assert abs(d["n_ionize_meta"] - do["n_ionize_meta"]) <= flips


def test_fp32_several_steps(pg):
    p = pic_inputs.params_rz32(gather=0)
    p.update(poisson_tol=1e-12, circuit_mode=1, Vs=400.0, Rext=2000.0, n_avg=4, gamma_i=0.2)
    p, parts = pic_inputs.seed_plasma(p, 32 * 32 * 8, seed=5, Te_eV=5.0)
    p, orc, h = _pair32(pg, p, parts)
    for _ in range(6):
        orc.step(1)
        pg.pic_step(h, 1)
    _check(pg, h, orc)


def test_fp32_set_get_roundtrip(pg):
    p = pic_inputs.params_rz32()
    p, parts = pic_inputs.seed_plasma(p, 50000, seed=9)
    p = pic_inputs.with_capacity(p, parts)
    h = pg.pic_create(dict(p, precision=1))
    pg.pic_set_particles(h, 0, 0, parts["e"])
    got = sort_by_id(pg.pic_get_particles(h, 0, 0))
    ref = sort_by_id(parts["e"])
    assert np.array_equal(got["id"], ref["id"])
    dr = p["R"] / p["nr"]
    assert np.abs(got["r"] - ref["r"]).max() <= 2.0 ** -23 * dr
    assert np.abs(got["z"] - ref["z"]).max() <= 2.0 ** -23 * p["L"] / p["nz"]
    for k in ("vr", "vt", "vz"):
        np.testing.assert_allclose(got[k], ref[k], rtol=2.0 ** -23)


def test_fp32_checkpoint_resume(pg, tmp_path):
    p = pic_inputs.params_rz32()
    p.update(circuit_mode=1, Vs=400.0, Rext=500.0, gamma_i=0.3, precision=1)
    p, parts = busy_state(p, ppc=8, seed=17)
    p = pic_inputs.with_capacity(p, parts, factor=2.0)
    h = pg.pic_create(p)
    for k, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, 0, sp, parts[k])
    pg.pic_solve_fields(h, 0)
    pg.pic_step(h, 3)
    pg.pic_save(h, 0, str(tmp_path / "ck32.bin"))
    pg.pic_step(h, 3)
    ref = [sort_by_id(pg.pic_get_particles(h, 0, sp)) for sp in (0, 1)]
    h2 = pg.pic_create(p)
    pg.pic_load(h2, 0, str(tmp_path / "ck32.bin"))
    pg.pic_step(h2, 3)
    for sp in (0, 1):
        got = sort_by_id(pg.pic_get_particles(h2, 0, sp))
        assert np.array_equal(got["id"], ref[sp]["id"])
        for k in ("r", "z", "vr", "vt", "vz"):
            scale = np.abs(ref[sp][k]).max()
            assert np.abs(got[k] - ref[sp][k]).max() <= 1e-5 * scale, (sp, k)
    assert pg.pic_diagnostics(h2, 0)["step"] == pg.pic_diagnostics(h, 0)["step"]


def test_fp32_diagnostics_vs_fp64_oracle(pg):
    """Diagnostics of 20 FP32 steps against the FP64 oracle from the same
    state; the errors are printed (they are quoted in the design notes)."""
    p = pic_inputs.params_rz32(gather=0)
    p.update(poisson_tol=1e-12, circuit_mode=1, Vs=400.0, Rext=200.0, n_avg=5)
    p, parts = pic_inputs.seed_plasma(p, 32 * 32 * 16, seed=23, Te_eV=3.0)
    p, orc, h = _pair32(pg, p, parts)
    errs = {k: 0.0 for k in ("I_cath", "V_cath", "n_e_peak", "n_i_peak", "W_field", "K_e", "K_i")}
    for _ in range(20):
        orc.step(1)
        pg.pic_step(h, 1)
        d, do = pg.pic_diagnostics(h, 0), orc.diag()
        for k in errs:
            den = max(abs(do[k]), 1e-30)
            errs[k] = max(errs[k], abs(d[k] - do[k]) / den)
    print("FP32 diagnostics, max relative error over 20 steps:", errs)
    for k, v in errs.items():
        assert v <= 1e-4, (k, v)


def test_fp32_reweight_keeps_the_oracles_particles(pg):
    """Re-weighting in FP32 mode draws from the particle ids alone, so it keeps
    exactly the oracle's set; the step after it matches at the FP32 bar with
    the tripled weight (charge Q included)."""
    p = pic_inputs.params_rz32()
    p.update(gamma_i=0.3, poisson_tol=1e-12, circuit_mode=1, Vs=400.0, Rext=100.0, n_avg=3)
    p, parts = busy_state(p, ppc=24, seed=43)
    p, orc, h = _pair32(pg, p, parts)
    pg.pic_reweight(h, 0, 3)
    orc.reweight(3)
    for sp in (0, 1):
        a = sort_by_id(pg.pic_get_particles(h, 0, sp))
        b = sort_by_id(orc.get_particles(sp))
        assert np.array_equal(a["id"], b["id"]), sp
    orc.step(1)
    pg.pic_step(h, 1)
    _check(pg, h, orc)
    assert pg.pic_diagnostics(h, 0)["weight"] == orc.weight == 3 * p["weight"]
    pg.pic_destroy(h)


def test_fp32_insulating_block(pg):
    p = pic_inputs.params_rz32()
    p.update(gap_neumann=1, wall_neumann=1, Rc=0.6 * p["R"], gamma_i=0.3, poisson_tol=1e-12,
             circuit_mode=1, Vs=400.0, Rext=100.0, n_avg=3)
    p, parts = busy_state(p, ppc=16, seed=57)
    p, orc, h = _pair32(pg, p, parts)
    orc.step(1)
    pg.pic_step(h, 1)
    _check(pg, h, orc)
    pg.pic_destroy(h)


def test_fp32_region_diagnostics(pg):
    """FP32 mode: the same region evaluation over FP32 records; temperatures
    and the ion histogram's total agree with the FP64 oracle at the FP32
    level."""
    p = pic_inputs.params_rz32()
    p.update(gamma_i=0.2, poisson_tol=1e-12, circuit_mode=1, Vs=400.0, Rext=100.0, n_avg=3,
             band_r_lo=0.010, band_r_hi=0.015, ied_bins=64, ied_emax=256.0)
    p, parts = busy_state(p, ppc=16, seed=67)
    p, orc, h = _pair32(pg, p, parts)
    orc.step(1)
    pg.pic_step(h, 1)
    orc.region_sample()
    pg.pic_region_sample(h, 0)
    a, b = pg.pic_region_read(h, 0), orc.regions()
    assert a["samples"] == 1
    assert a["ion_impacts"] == b["ion_impacts"] > 0
    for k in range(3):
        if b["ncell"][k] > 0:
            assert a["Te"][k] == pytest.approx(b["Te"][k], rel=2e-3), k
    pg.pic_destroy(h)


def test_fp32_sort_every(pg):
    """FP32 records with a full sort every third step: dead records and
    appended births between sorts; after five steps the run is on the FP64
    oracle's track at the FP32 bar."""
    p = pic_inputs.params_rz32()
    p.update(gamma_i=0.3, poisson_tol=1e-12, circuit_mode=1, Vs=400.0, Rext=100.0, n_avg=3,
             sort_every=3)
    p, parts = busy_state(p, ppc=16, seed=83)
    p, orc, h = _pair32(pg, p, parts)
    for _ in range(5):
        orc.step(1)
        pg.pic_step(h, 1)
    _check(pg, h, orc)
    pg.pic_destroy(h)


@pytest.mark.parametrize("shape", [2, 3])
def test_fp32_tile_shapes(pg, shape):
    """FP32 records on the 16 x 8 and 8 x 16 cell tiles (the sort key and the
    deposit patch of that shape, a full sort every third step): on the FP64
    oracle's track at the FP32 bar after five steps."""
    p = pic_inputs.params_rz32()
    p.update(gamma_i=0.3, poisson_tol=1e-12, circuit_mode=1, Vs=400.0, Rext=100.0, n_avg=3,
             sort_every=3)
    p, parts = busy_state(p, ppc=16, seed=85 + shape)
    p, orc, h = _pair32(pg, p, parts)
    pg.pic_set_tile(h, shape)
    for _ in range(5):
        orc.step(1)
        pg.pic_step(h, 1)
    assert pg.pic_tuned_tile(h) == shape
    _check(pg, h, orc)
    pg.pic_destroy(h)
