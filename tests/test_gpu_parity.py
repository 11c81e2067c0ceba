"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on
identical seeded states, one step and several steps, element by element.

Bar (FP64 mode): positions and velocities per species within
||a - b||_inf / ||b||_inf <= 1e-12 with identical id sets; phi within 1e-10
of the oracle's; integer outputs (particle counts, cathode impacts,
secondary electrons, collision counts) equal.
"""
import numpy as np
import pytest

import oracle
import pic_inputs
from parity import (FIELD_TOL, PARTICLE_TOL, busy_state, check_step64, compare_species,
                    field_err, sort_by_id)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_10727_gb300 as pg
    import torch
    assert torch.cuda.is_available()
    return pg


def _pair(pg, p, parts, set_phi=True):
    p = pic_inputs.with_capacity(p, parts, factor=2.0)
    orc = oracle.Oracle(p, parts)
    h = pg.pic_create(p)
    for k, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, 0, sp, parts[k])
    if set_phi:
        pg.pic_set_phi(h, 0, orc.fields()["phi"])
    return p, orc, h


def _check_step(pg, h, orc, check_phi=True):
    return check_step64(pg, h, orc, 0, check_phi)


@pytest.mark.parametrize("gather", [0, 1])
@pytest.mark.parametrize("rweight", [0, 1])
def test_one_step_busy_state(pg, gather, rweight):
    p = pic_inputs.params_rz32(gather=gather)
    p.update(rweight=rweight, gamma_i=0.5, gamma_e=0.3, poisson_tol=1e-13,
             circuit_mode=1, Vs=400.0, Rext=100.0, n_avg=3)
    p, parts = busy_state(p, ppc=16, seed=3 + gather + 2 * rweight)
    p, orc, h = _pair(pg, p, parts)
    orc.step(1)
    pg.pic_step(h, 1)
    d = _check_step(pg, h, orc)
    # the state does exercise every branch
    assert d["n_sey"] > 0 and d["n_ionize"] > 0 and d["n_excite"] > 0 and d["n_e_cath"] > 0
    assert pg.pic_get_next_id(h, 0) == orc.next_id


@pytest.mark.parametrize("gather", [0, 1])
def test_collision_queue_overflow(pg, gather):
    """A collision-dominated gas (200 x the density: p_null about 0.83): in the
    first step's 1024-particle chunks more electrons are collision candidates
    than the per-chunk queue holds (512), so the rest run from the per-thread
    masks after the queue; the step still matches the oracle."""
    p = pic_inputs.params_rz32(gather=gather)
    p.update(n_gas=200.0 * p["n_gas"], poisson_tol=1e-13, circuit_mode=1, Vs=400.0, Rext=100.0,
             n_avg=3)
    p, parts = busy_state(p, ppc=16, seed=43 + gather)
    p, orc, h = _pair(pg, p, parts)
    orc.step(1)
    pg.pic_step(h, 1)
    d = _check_step(pg, h, orc)
    assert d["n_elastic"] + d["n_excite"] + d["n_ionize"] > 2048


@pytest.mark.parametrize("gather", [0, 1])
def test_metastable_ionization_and_electron_sey(pg, gather):
    """Reaction (1d) off an Ar* background (dense here, 3e20 m^-3, so that a
    step has tens of events) and electron-induced secondary emission at the
    paper's gamma_e = 0.1 (Section 3)."""
    p = pic_inputs.params_rz32(gather=gather)
    p.update(n_meta=3e20, gamma_i=0.2, gamma_e=0.1, poisson_tol=1e-13, circuit_mode=1,
             Vs=400.0, Rext=100.0, n_avg=3)
    p, parts = busy_state(p, ppc=16, seed=31 + gather)
    p, orc, h = _pair(pg, p, parts)
    for _ in range(2):
        orc.step(1)
        pg.pic_step(h, 1)
        d = _check_step(pg, h, orc)
    assert d["n_ionize_meta"] > 0 and d["n_e_cath"] > 0


def test_ragged_grid_and_counts(pg):
    # 20 x 36 cells: partial 8x8 tiles along both axes; particle counts not a
    # multiple of the push chunk
    p = pic_inputs.params_rz32(gather=0)
    p.update(nr=20, nz=36, R=0.02, L=0.03, Rc=0.012, gamma_i=0.5, poisson_tol=1e-13)
    p, parts = busy_state(p, ppc=7, seed=21)
    p, orc, h = _pair(pg, p, parts)
    for _ in range(3):
        orc.step(1)
        pg.pic_step(h, 1)
        _check_step(pg, h, orc)


@pytest.mark.parametrize("extrap", [0, 1])
@pytest.mark.parametrize("gather", [0, 1])
def test_several_steps_seed_plasma(pg, gather, extrap):
    p = pic_inputs.params_rz32(gather=gather)
    p.update(poisson_tol=1e-13, circuit_mode=1, Vs=400.0, Rext=2000.0, n_avg=4, gamma_i=0.2,
             phi_extrapolate=extrap)
    p, parts = pic_inputs.seed_plasma(p, 32 * 32 * 8, seed=5, Te_eV=5.0)
    p, orc, h = _pair(pg, p, parts)
    for _ in range(6):
        orc.step(1)
        pg.pic_step(h, 1)
        _check_step(pg, h, orc)


def test_solve_fields_matches_oracle(pg):
    p = pic_inputs.params_rz32()
    p.update(poisson_tol=1e-13)
    p, parts = busy_state(p, ppc=4, seed=8)
    p, orc, h = _pair(pg, p, parts, set_phi=False)
    pg.pic_solve_fields(h, 0)
    pg.pic_sync(h)
    fg, fo = pg.pic_get_fields(h, 0), orc.fields()
    assert field_err(fg["Q"], fo["Q"]) <= 1e-12
    assert field_err(fg["rho"], fo["rho"]) <= 1e-12
    assert field_err(fg["phi"], fo["phi"]) <= FIELD_TOL


@pytest.mark.parametrize("nr,nz", [(32, 32), (48, 20), (128, 128), (256, 256)])
def test_poisson_standalone(pg, nr, nz):
    import torch
    p = pic_inputs.params_rz256()
    p.update(nr=nr, nz=nz, R=0.05, L=0.05 * nz / nr)
    rng = np.random.default_rng(nr + nz)
    V = oracle.node_volume(p)
    rho = rng.normal(size=(nr + 1, nz + 1)) * 1e-6
    bc = np.zeros_like(rho)
    dr = p["R"] / nr
    mc = [m for m in range(nr) if m * dr <= 0.6 * p["R"]]
    bc[mc, 0] = -321.0
    bc[:, nz] = 5.0 * rng.random(nr + 1)
    bc[nr, :] = 2.0
    phi_o = oracle.poisson(p, rho, bc)
    Q = torch.tensor(rho * V, device="cuda")
    phi = torch.tensor(bc, device="cuda")
    rc, it, res = pg.pic_poisson_solve(nr, nz, p["R"], p["L"], 1e-13, 500, Q, phi)
    torch.cuda.synchronize()
    assert rc == 0 and res <= 1e-13, (rc, it, res)
    assert field_err(phi.cpu().numpy(), phi_o) <= FIELD_TOL
    # Dirichlet nodes untouched
    out = phi.cpu().numpy()
    assert np.array_equal(out[:, 0], bc[:, 0]) and np.array_equal(out[nr, :], bc[nr, :])


def test_determinism_and_checkpoint(pg, tmp_path):
    p = pic_inputs.params_rz32()
    p.update(circuit_mode=1, Vs=400.0, Rext=500.0, gamma_i=0.3)
    p, parts = busy_state(p, ppc=8, seed=13)
    p = pic_inputs.with_capacity(p, parts, factor=2.0)
    runs = []
    for _ in range(2):
        h = pg.pic_create(p)
        for k, sp in (("e", 0), ("i", 1)):
            pg.pic_set_particles(h, 0, sp, parts[k])
        pg.pic_solve_fields(h, 0)
        pg.pic_step(h, 4)
        pg.pic_save(h, 0, str(tmp_path / "ck.bin"))
        pg.pic_step(h, 4)
        runs.append((h, [sort_by_id(pg.pic_get_particles(h, 0, sp)) for sp in (0, 1)],
                     pg.pic_get_fields(h, 0)["phi"], pg.pic_diagnostics(h, 0)))
    (_, pa, fa, da), (_, pb, fb, db) = runs
    for sp in (0, 1):
        for k in pa[sp]:
            assert np.array_equal(pa[sp][k], pb[sp][k]), (sp, k)
    assert np.array_equal(fa, fb)
    # resume from the checkpoint in a fresh handle: identical continuation
    h2 = pg.pic_create(p)
    pg.pic_load(h2, 0, str(tmp_path / "ck.bin"))
    pg.pic_step(h2, 4)
    for sp in (0, 1):
        pc = sort_by_id(pg.pic_get_particles(h2, 0, sp))
        for k in pc:
            assert np.array_equal(pc[k], pa[sp][k]), (sp, k)
    assert np.array_equal(pg.pic_get_fields(h2, 0)["phi"], fa)
    dc = pg.pic_diagnostics(h2, 0)
    assert dc["step"] == da["step"] and dc["V_cath"] == da["V_cath"]


def test_edge_cases(pg):
    p = pic_inputs.params_rz32()
    p.update(cap_e=4096, cap_i=4096, birth_cap=1024)
    empty = {k: np.zeros(0) for k in ("r", "z", "vr", "vt", "vz")} | {"id": np.zeros(0, np.int64)}
    # empty plasma: steps run, fields are the vacuum solution
    h = pg.pic_create(p)
    pg.pic_solve_fields(h, 0)
    pg.pic_step(h, 3)
    d = pg.pic_diagnostics(h, 0)
    assert d["N_e"] == 0 and d["N_i"] == 0 and d["status"] == 0
    orc = oracle.Oracle(p, {"e": empty, "i": empty})
    orc.step(3)
    assert field_err(pg.pic_get_fields(h, 0)["phi"], orc.fields()["phi"]) <= FIELD_TOL
    # every particle leaves in one step
    n = 1000
    gone = {"r": np.full(n, 0.01), "z": np.full(n, p["L"] * 0.999), "vr": np.zeros(n),
            "vt": np.zeros(n), "vz": np.full(n, 1e7), "id": np.arange(n)}
    h = pg.pic_create(p)
    pg.pic_set_particles(h, 0, 0, gone)
    pg.pic_step(h, 1)
    assert pg.pic_count(h, 0, 0) == 0
    # out-of-domain input is rejected
    bad = dict(gone, r=np.full(n, 2 * p["R"]))
    h = pg.pic_create(p)
    with pytest.raises(pg.PicError) as ei:
        pg.pic_set_particles(h, 0, 0, bad)
    assert ei.value.code == -5
    # more particles than the capacity
    h = pg.pic_create(p)
    big = {k: np.resize(v, 5000) for k, v in gone.items()}
    big["id"] = np.arange(5000)
    with pytest.raises(pg.PicError) as ei:
        pg.pic_set_particles(h, 0, 0, big)
    assert ei.value.code == -3


def test_capacity_and_nonconvergence_latch(pg):
    p = pic_inputs.params_rz32()
    p, parts = busy_state(p, ppc=4, seed=2)
    p = pic_inputs.with_capacity(p, parts, factor=1.0)
    p["birth_cap"] = 1          # more than one birth in the first step
    h = pg.pic_create(p)
    for k, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, 0, sp, parts[k])
    pg.pic_step(h, 2)
    with pytest.raises(pg.PicError) as ei:
        pg.pic_sync(h)
    assert ei.value.code == -3
    q = dict(p, birth_cap=100000, poisson_max_iter=1, poisson_tol=1e-15)
    h = pg.pic_create(q)
    for k, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, 0, sp, parts[k])
    pg.pic_solve_fields(h, 0)
    with pytest.raises(pg.PicError) as ei:
        pg.pic_sync(h)
    assert ei.value.code == -4


def test_graph_replay_matches_oracle(pg):
    """On a side stream pic_step captures one step into a CUDA graph and
    replays it; the replayed steps match the oracle like eager ones."""
    import torch
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        p = pic_inputs.params_rz32(gather=0)
        p.update(gamma_i=0.5, poisson_tol=1e-13, circuit_mode=1, Vs=400.0, Rext=100.0, n_avg=3)
        p, parts = busy_state(p, ppc=8, seed=41)
        p, orc, h = _pair(pg, p, parts)
        # the first four steps tune the push's chunk size and the next two the
        # other cell tile shapes (eager launches; a shape trial re-sorts the
        # particles first), later ones replay the captured step
        for k in range(8):
            orc.step(1)
            pg.pic_step(h, 1)
            assert pg.pic_uses_graph(h) == (k >= 6)
            _check_step(pg, h, orc)
        assert pg.pic_tuned_chunk(h) in (4, 8, 16, 32)
        assert pg.pic_tuned_tile(h) in (1, 2, 3)
    side.synchronize()


@pytest.mark.parametrize("gather", [0, 1])
def test_reweight_matches_oracle(pg, gather, tmp_path):
    """Re-weighting between steps (Section 6): the same particles kept as the
    oracle's (per-id draw), weight x 3, then steps that match the oracle's
    with the new weight; a checkpoint taken after it restores the weight."""
    p = pic_inputs.params_rz32(gather=gather)
    p.update(gamma_i=0.3, gamma_e=0.1, poisson_tol=1e-13, circuit_mode=1, Vs=400.0,
             Rext=100.0, n_avg=3)
    p, parts = busy_state(p, ppc=24, seed=41 + gather)
    p, orc, h = _pair(pg, p, parts)
    for _ in range(2):
        orc.step(1)
        pg.pic_step(h, 1)
    d0 = _check_step(pg, h, orc)
    assert d0["ppc_max_e"] > 0 and d0["ppc_max_i"] > 0
    n_before = [pg.pic_count(h, 0, sp) for sp in (0, 1)]
    pg.pic_reweight(h, 0, 3)
    orc.reweight(3)
    for sp in (0, 1):
        a = sort_by_id(pg.pic_get_particles(h, 0, sp))
        b = sort_by_id(orc.get_particles(sp))
        assert np.array_equal(a["id"], b["id"]), sp
        # binomial(n, 1/3) at 5 sigma
        n = n_before[sp]
        assert abs(a["id"].size - n / 3) < 5 * np.sqrt(n * 2 / 9)
    pg.pic_save(h, 0, str(tmp_path / "rw.bin"))
    for _ in range(3):
        orc.step(1)
        pg.pic_step(h, 1)
        d = _check_step(pg, h, orc)
    assert d["weight"] == orc.weight == 3 * p["weight"]
    # resume from the checkpoint in a fresh handle created with the old weight
    h2 = pg.pic_create(p)
    pg.pic_load(h2, 0, str(tmp_path / "rw.bin"))
    pg.pic_step(h2, 3)
    d2 = pg.pic_diagnostics(h2, 0)
    assert d2["weight"] == 3 * p["weight"]
    for sp in (0, 1):
        a = sort_by_id(pg.pic_get_particles(h2, 0, sp))
        b = sort_by_id(pg.pic_get_particles(h, 0, sp))
        for k in a:
            assert np.array_equal(a[k], b[k]), (sp, k)
    assert d2["I_cath"] == d["I_cath"]
    assert d2["K_e"] == pytest.approx(d["K_e"], rel=1e-12)   # atomic summation order
    pg.pic_destroy(h2)
    pg.pic_destroy(h)


def test_reweight_factor_checks_and_graph(pg):
    """Argument checks; on a side stream the captured step is dropped by the
    re-weighting and captured again, and the replayed steps match the oracle
    with the new weight."""
    import torch
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        p = pic_inputs.params_rz32()
        p.update(gamma_i=0.3, poisson_tol=1e-13, circuit_mode=1, Vs=400.0, Rext=100.0, n_avg=3)
        p, parts = busy_state(p, ppc=12, seed=5)
        p, orc, h = _pair(pg, p, parts)
        with pytest.raises(pg.PicError):
            pg.pic_reweight(h, 0, 0)
        n0 = pg.pic_count(h, 0, 0)
        pg.pic_reweight(h, 0, 1)
        assert pg.pic_count(h, 0, 0) == n0
        for _ in range(7):    # six tuning steps, then the captured step
            orc.step(1)
            pg.pic_step(h, 1)
        assert pg.pic_uses_graph(h) == 1
        pg.pic_reweight(h, 0, 2)
        orc.reweight(2)
        assert pg.pic_uses_graph(h) == 0
        for _ in range(2):
            orc.step(1)
            pg.pic_step(h, 1)
            assert pg.pic_uses_graph(h) == 1
            _check_step(pg, h, orc)
        pg.pic_destroy(h)


@pytest.mark.parametrize("nr,nz,gap,wall", [(32, 32, 1, 0), (32, 32, 1, 1), (48, 20, 0, 1),
                                            (128, 128, 1, 1), (256, 256, 1, 0)])
def test_poisson_insulating_boundaries(pg, nr, nz, gap, wall):
    """Standalone solve with the insulating block (Section 3: Neumann) on
    z = 0 outside the cathode and / or on the wall r = R, against the oracle's
    direct solve of the same finite-volume system."""
    import torch
    p = pic_inputs.params_rz256()
    p.update(nr=nr, nz=nz, R=0.05, L=0.05 * nz / nr, Rc=0.6 * 0.05, gap_neumann=gap,
             wall_neumann=wall)
    rng = np.random.default_rng(nr + 3 * nz + gap + 2 * wall)
    V = oracle.node_volume(p)
    rho = rng.normal(size=(nr + 1, nz + 1)) * 1e-6
    bc = np.zeros_like(rho)
    dr = p["R"] / nr
    mc = [m for m in range(nr) if m * dr <= p["Rc"]]
    bc[mc, 0] = -321.0
    bc[:, nz] = 5.0 * rng.random(nr + 1)
    bc[nr, :] = 2.0
    phi_o = oracle.poisson(p, rho, bc)
    g = len(mc) if gap else nr + 1
    Q = torch.tensor(rho * V, device="cuda")
    phi = torch.tensor(bc, device="cuda")
    rc, it, res = pg.pic_poisson_solve(nr, nz, p["R"], p["L"], 1e-13, 500, Q, phi,
                                       first_insulating_z0=g, wall_insulating=wall)
    torch.cuda.synchronize()
    assert rc == 0 and res <= 1e-13, (rc, it, res)
    out = phi.cpu().numpy()
    assert field_err(out, phi_o) <= FIELD_TOL
    # conductor nodes untouched; insulating nodes solved (they differ from bc)
    assert np.array_equal(out[mc, 0], bc[mc, 0]) and np.array_equal(out[:, nz], bc[:, nz])
    if gap:
        assert not np.array_equal(out[len(mc):nr, 0], bc[len(mc):nr, 0])
    if wall:
        assert not np.array_equal(out[nr, 1:nz], bc[nr, 1:nz])
    else:
        assert np.array_equal(out[nr, :], bc[nr, :])


@pytest.mark.parametrize("gather", [0, 1])
@pytest.mark.parametrize("wall", [0, 1])
def test_insulating_block_steps_match_oracle(pg, gather, wall):
    """Full steps with the paper's boundary (Section 3): the z = 0 plane beside
    the cathode insulating (and the wall r = R in the second reading)."""
    p = pic_inputs.params_rz32(gather=gather)
    p.update(gap_neumann=1, wall_neumann=wall, Rc=0.6 * p["R"], gamma_i=0.3, gamma_e=0.1,
             poisson_tol=1e-13, circuit_mode=1, Vs=400.0, Rext=100.0, n_avg=3)
    p, parts = busy_state(p, ppc=16, seed=51 + gather + 2 * wall)
    p, orc, h = _pair(pg, p, parts)
    for _ in range(3):
        orc.step(1)
        pg.pic_step(h, 1)
        _check_step(pg, h, orc)
    phi = pg.pic_get_fields(h, 0)["phi"]
    m_gap = int(0.6 * p["nr"]) + 2
    assert phi[m_gap, 0] != 0.0          # the block floats
    pg.pic_destroy(h)


def _fast_cathode_ions(p, parts, seed):
    """The cathode-bound ions of busy_state given a spread of energies
    (about 20 to 330 eV) so that the ion energy histogram has many bins."""
    rng = np.random.default_rng(seed)
    i = parts["i"]
    k = np.flatnonzero(i["vz"] == -2e4)
    vz = -rng.uniform(1.0e4, 4.0e4, k.size)
    i["vz"][k] = vz
    i["z"][k] = rng.random(k.size) * np.abs(vz) * p["dt"]


@pytest.mark.parametrize("gather", [0, 1])
def test_region_diagnostics_match_oracle(pg, gather):
    """Region diagnostics (Sections 4, 5, 7): per-column sheath and bulk
    edges, electron temperatures by region and the cathode ion energy
    histogram accumulated over three steps, against the oracle's."""
    p = pic_inputs.params_rz32(gather=gather)
    p.update(gamma_i=0.2, poisson_tol=1e-13, circuit_mode=1, Vs=400.0, Rext=100.0, n_avg=3,
             band_r_lo=0.010, band_r_hi=0.015, ied_bins=64, ied_emax=256.0)
    p, parts = busy_state(p, ppc=16, seed=61 + gather)
    _fast_cathode_ions(p, parts, 7 + gather)
    p, orc, h = _pair(pg, p, parts)
    for _ in range(3):
        orc.step(1)
        pg.pic_step(h, 1)
        orc.region_sample()
        pg.pic_region_sample(h, 0)
    _check_step(pg, h, orc)
    a, b = pg.pic_region_read(h, 0), orc.regions()
    bh, bo = orc.ied()
    assert a["samples"] == b["samples"] == 3
    assert np.array_equal(a["zs"], b["zs"]) and np.array_equal(a["zb"], b["zb"])
    assert a["ncell"] == b["ncell"] and sum(a["ncell"]) > 0
    for k in range(3):
        assert a["Te"][k] == pytest.approx(b["Te"][k], rel=1e-10), k
    assert a["z_sheath"] == pytest.approx(b["z_sheath"], rel=1e-14)
    assert a["z_bulk"] == pytest.approx(b["z_bulk"], rel=1e-14)
    assert np.array_equal(a["ied"], bh) and a["ied_overflow"] == bo
    assert a["ion_impacts"] == b["ion_impacts"] > 50
    assert np.count_nonzero(bh) > 10
    pg.pic_region_reset(h, 0)
    z = pg.pic_region_read(h, 0)
    assert z["samples"] == 0 and z["ion_impacts"] == 0 and z["ncell"] == [0, 0, 0]
    pg.pic_destroy(h)


@pytest.mark.parametrize("extrap", [0, 1])
@pytest.mark.parametrize("gather", [0, 1])
def test_sort_every_matches_oracle(pg, gather, extrap, tmp_path):
    """Full cell sorts only every third step (dead slots and appended births in
    between): the step's results do not depend on the particle order, so the
    run matches the oracle as with a sort every step -- integer counters every
    step (no compaction), particles and fields at the end; a checkpoint taken
    between sorts resumes identically."""
    p = pic_inputs.params_rz32(gather=gather)
    p.update(gamma_i=0.3, gamma_e=0.1, poisson_tol=1e-13, circuit_mode=1, Vs=400.0,
             Rext=100.0, n_avg=3, sort_every=3, phi_extrapolate=extrap)
    p, parts = busy_state(p, ppc=16, seed=71 + gather)
    p, orc, h = _pair(pg, p, parts)
    for k in range(7):
        orc.step(1)
        pg.pic_step(h, 1)
        de, do = pg.pic_diagnostics(h, 0), orc.diag()
        for key in ("N_e", "N_i", "n_ion_cath", "n_e_cath", "n_sey", "n_ionize", "n_excite",
                    "n_elastic"):
            assert de[key] == do[key], (k, key)
        if k == 3:   # between sorts (steps 2 and 5 sort): checkpoint, compacting
            pg.pic_save(h, 0, str(tmp_path / "mid.bin"))
    _check_step(pg, h, orc)
    h2 = pg.pic_create(p)
    pg.pic_load(h2, 0, str(tmp_path / "mid.bin"))
    pg.pic_step(h2, 3)
    for sp in (0, 1):
        a = sort_by_id(pg.pic_get_particles(h2, 0, sp))
        b = sort_by_id(pg.pic_get_particles(h, 0, sp))
        for q in a:
            assert np.array_equal(a[q], b[q]), (sp, q)
    assert pg.pic_diagnostics(h2, 0)["particle_steps"] == pg.pic_diagnostics(h, 0)["particle_steps"]
    pg.pic_destroy(h2)
    pg.pic_destroy(h)


def test_sort_every_graph_and_reads_between_sorts(pg):
    """With the step captured in a CUDA graph and sorts every fourth step,
    reads between sorts (count, particles, region sample, re-weighting)
    compact the arrays and leave the run on the oracle's track."""
    import torch
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        p = pic_inputs.params_rz32()
        p.update(gamma_i=0.3, poisson_tol=1e-13, circuit_mode=1, Vs=400.0, Rext=100.0, n_avg=3,
                 sort_every=4, ied_bins=16, ied_emax=512.0)
        p, parts = busy_state(p, ppc=12, seed=81)
        p, orc, h = _pair(pg, p, parts)
        pg.pic_step(h, 7)     # six tuning steps (each sorts), then the captured step
        orc.step(7)
        assert pg.pic_uses_graph(h) == 1
        assert pg.pic_count(h, 0, 0) == orc.count(0)       # compacts (step 7: unsorted)
        pg.pic_region_sample(h, 0)
        pg.pic_step(h, 2)
        orc.step(2)
        pg.pic_reweight(h, 0, 2)
        orc.reweight(2)
        pg.pic_step(h, 3)
        orc.step(3)
        _check_step(pg, h, orc)
        pg.pic_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_pinned_host_upload_equals_pageable(pg, precision):
    """Pinned host arrays are read in place by the kernels; the loaded state is
    the one the copy path (pageable arrays) gives, bit for bit."""
    import ctypes as C
    import torch
    p = pic_inputs.params_rz32(precision=precision)
    p, parts = busy_state(p, ppc=9, seed=91)
    p = pic_inputs.with_capacity(p, parts, factor=2.0)
    ha, hb = pg.pic_create(p), pg.pic_create(p)
    lib = pg.load_library()
    for k, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(ha, 0, sp, parts[k])                    # pageable numpy arrays
        t = {q: torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for q, a in parts[k].items()}
        rc = lib.pic_set_particles(hb.ptr, 0, sp, t["r"].numel(), t["r"].data_ptr(),
                                   t["z"].data_ptr(), t["vr"].data_ptr(), t["vt"].data_ptr(),
                                   t["vz"].data_ptr(), t["id"].data_ptr(), 0)
        assert rc == 0
    for sp in (0, 1):
        a = sort_by_id(pg.pic_get_particles(ha, 0, sp))
        b = sort_by_id(pg.pic_get_particles(hb, 0, sp))
        for q in a:
            assert np.array_equal(a[q], b[q]), (sp, q)
    pg.pic_destroy(ha)
    pg.pic_destroy(hb)


def test_phi_extrapolation_same_phi_fewer_iterations(pg):
    """Each step's Poisson solve started from 2 phi^(n-1) - phi^(n-2) on the
    unknown nodes: the first step after pic_solve_fields has no earlier
    solution and is the plain step bit for bit (2 phi - phi = phi exactly);
    on the second both starts reach a 1e-13 relative residual, so with the
    condition number of the 32 x 32 operator (below 1e4) the two phi agree to
    1e-10; over the run the extrapolated starts need no more multigrid-PCG
    iterations than the previous solution as the start."""
    p = pic_inputs.params_rz32()
    p.update(circuit_mode=1, Vs=400.0, Rext=2000.0, n_avg=4, poisson_tol=1e-13,
             poisson_precond=1, poisson_max_iter=400)
    p, parts = busy_state(p, ppc=32, seed=23)
    p = pic_inputs.with_capacity(p, parts, factor=2.0)
    hs = []
    for ex in (0, 1):
        h = pg.pic_create(dict(p, phi_extrapolate=ex))
        for k, sp in (("e", 0), ("i", 1)):
            pg.pic_set_particles(h, 0, sp, parts[k])
        pg.pic_solve_fields(h, 0)
        hs.append(h)
    iters = [[], []]
    for step in range(30):
        for j, h in enumerate(hs):
            pg.pic_step(h, 1)
            iters[j].append(pg.pic_diagnostics(h, 0)["poisson_iters"])
        phi0, phi1 = (pg.pic_get_fields(h, 0)["phi"] for h in hs)
        if step == 0:
            assert np.array_equal(phi0, phi1)
        elif step == 1:
            assert field_err(phi1, phi0) <= FIELD_TOL
    print(f"Poisson iterations over 30 steps: start phi^(n-1) {sum(iters[0])}, "
          f"extrapolated {sum(iters[1])}")
    assert iters[0][0] == iters[1][0]
    assert sum(iters[1]) <= sum(iters[0])
    for h in hs:
        pg.pic_destroy(h)


@pytest.mark.parametrize("gather", [0, 1])
def test_sine_transform_and_multigrid_preconditioners_agree(pg, gather):
    """The two preconditioners of the PCG solve (Section 3's Poisson problem
    with every boundary node a conductor): the sine transform along z with a
    tridiagonal solve per mode is exact for the operator up to its FP32
    arithmetic, the multigrid V-cycle is not; both solve to the same relative
    residual, so over several steps the particles and phi of the two runs
    match the oracle, and the sine-transform runs need at most three
    iterations per step."""
    p = pic_inputs.params_rz32(gather=gather)
    p.update(poisson_tol=1e-13, circuit_mode=1, Vs=400.0, Rext=2000.0, n_avg=4, gamma_i=0.2)
    p, parts = pic_inputs.seed_plasma(p, 32 * 32 * 8, seed=19, Te_eV=5.0)
    p = pic_inputs.with_capacity(p, parts, factor=2.0)
    orc = oracle.Oracle(p, parts)
    hs = []
    for pre in (0, 1):
        h = pg.pic_create(dict(p, poisson_precond=pre))
        for k, sp in (("e", 0), ("i", 1)):
            pg.pic_set_particles(h, 0, sp, parts[k])
        pg.pic_set_phi(h, 0, orc.fields()["phi"])
        hs.append(h)
    iters = [0, 0]
    for _ in range(4):
        orc.step(1)
        for j, h in enumerate(hs):
            pg.pic_step(h, 1)
            d = check_step64(pg, h, orc)
            iters[j] = max(iters[j], d["poisson_iters"])
            assert d["poisson_resid"] <= 1e-13
    print(f"most PCG iterations per step: sine transform {iters[0]}, multigrid {iters[1]}")
    assert iters[0] <= 3 and iters[0] < iters[1]
    for h in hs:
        pg.pic_destroy(h)


@pytest.mark.parametrize("nr, nz", [(256, 256), (256, 512), (128, 128), (20, 36), (320, 64),
                                    (40, 26)])
def test_sine_transform_solve_fields(pg, nr, nz):
    """pic_solve_fields on the sine-transform preconditioner against the
    oracle's banded Cholesky solve, on the benchmark grids and ragged ones:
    three rows per block with a shorter last block (320 rows over at most one
    block per SM), transform rows of 7 or 9 float4 columns whose n-range parts
    leave threads of the block idle (25 and 35 modes)."""
    p = pic_inputs.params_rz256()
    p.update(nr=nr, nz=nz, L=p["R"] * nz / nr, poisson_tol=1e-13)
    p, parts = pic_inputs.grown_ring_state(p, 20 * nr * nz, seed=nr + nz)
    p = pic_inputs.with_capacity(p, parts)
    orc = oracle.Oracle(p, parts)
    h = pg.pic_create(p)
    for k, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, 0, sp, parts[k])
    pg.pic_solve_fields(h, 0)
    assert field_err(pg.pic_get_fields(h, 0)["phi"], orc.fields()["phi"]) <= FIELD_TOL
    pg.pic_set_chunk(h, 8)
    pg.pic_step(h, 1)
    d = pg.pic_diagnostics(h, 0)
    assert d["poisson_iters"] <= 3 and d["poisson_resid"] <= 1e-13
    pg.pic_destroy(h)


@pytest.mark.parametrize("gather", [0, 1])
def test_tile_shapes_match_oracle(pg, gather):
    """The cell tile shape (8 x 8, 16 x 8, 8 x 16) changes the particles' sort
    order and the push's deposit patch, not the results: with a full sort every
    third step (dead slots and appended births in between) and the shape
    switched between steps (the particles re-sorted by the new keys, mid-way
    between two sorts), every step's counters and the final particles and
    fields match the oracle at the FP64 bar, on a ragged 20 x 36 grid whose
    tiles are partly outside it."""
    p = pic_inputs.params_rz32(gather=gather)
    p.update(nr=20, nz=36, L=p["R"] * 36 / 20, gamma_i=0.3, gamma_e=0.1, poisson_tol=1e-13,
             circuit_mode=1, Vs=400.0, Rext=100.0, n_avg=3, sort_every=3)
    p, parts = busy_state(p, ppc=16, seed=91 + gather)
    p, orc, h = _pair(pg, p, parts)
    pg.pic_set_chunk(h, 4)
    for k, shape in enumerate((2, 2, 3, 3, 1, 2, 3)):
        pg.pic_set_tile(h, shape)
        assert pg.pic_tuned_tile(h) == shape
        orc.step(1)
        pg.pic_step(h, 1)
        de, do = pg.pic_diagnostics(h, 0), orc.diag()
        for key in ("N_e", "N_i", "n_ion_cath", "n_e_cath", "n_sey", "n_ionize", "n_excite",
                    "n_elastic"):
            assert de[key] == do[key], (k, shape, key)
    _check_step(pg, h, orc)
    pg.pic_destroy(h)
