"""The batched ensemble (one handle, several independent discharges) against
the same discharges run one by one.

In FP64 mode every result of a step is independent of the order in which the
particles are processed (the deposit is an exact integer sum, births are
ordered by parent id), so the ensemble must reproduce the single-instance runs
bit for bit -- including while the autotuner switches chunk sizes and after
the step is captured into a CUDA graph.  The single-instance path is itself
checked against the oracle in test_gpu_parity.py; instance 0's first step is
checked against the oracle here as well.
"""
import numpy as np
import pytest

import oracle
import pic_inputs
from parity import PARTICLE_TOL, busy_state, compare_species, sort_by_id

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_10727_gb300 as pg
    return pg


def _instances(precision=0):
    out = []
    for k, (gamma, rext, ppc) in enumerate([(0.05, 50.0, 3), (0.1, 100.0, 9), (0.2, 200.0, 5),
                                            (0.3, 400.0, 14)]):
        p = pic_inputs.params_rz32(gather=0, precision=precision)
        p.update(nr=32, nz=48, R=0.02, L=0.03, Rc=0.015, gamma_i=gamma, circuit_mode=1,
                 Vs=400.0, Rext=rext, n_avg=4, seed=7 + k, poisson_tol=1e-12)
        p, parts = busy_state(p, ppc=ppc, seed=100 + k)
        p = pic_inputs.with_capacity(p, parts, factor=2.0)
        out.append((p, parts))
    return out


def _load(pg, h, k, parts):
    for key, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, k, sp, parts[key])


@pytest.mark.parametrize("side_stream", [False, True])
def test_ensemble_equals_individual_runs(pg, side_stream):
    import torch
    insts = _instances()
    steps = 7
    stream = torch.cuda.Stream() if side_stream else torch.cuda.current_stream()
    with torch.cuda.stream(stream):
        ens = pg.pic_create([p for p, _ in insts])
        for k, (p, parts) in enumerate(insts):
            _load(pg, ens, k, parts)
            pg.pic_solve_fields(ens, k)
        pg.pic_step(ens, steps)
        pg.pic_sync(ens)
        assert pg.pic_tuned_chunk(ens) in (4, 8, 16, 32)
        if side_stream:
            assert pg.pic_uses_graph(ens)
        for k, (p, parts) in enumerate(insts):
            one = pg.pic_create(p)
            _load(pg, one, 0, parts)
            pg.pic_solve_fields(one, 0)
            pg.pic_step(one, steps)
            for sp in (0, 1):
                a = sort_by_id(pg.pic_get_particles(ens, k, sp))
                b = sort_by_id(pg.pic_get_particles(one, 0, sp))
                for q in a:
                    assert np.array_equal(a[q], b[q]), (k, sp, q)
            fa, fb = pg.pic_get_fields(ens, k), pg.pic_get_fields(one, 0)
            assert np.array_equal(fa["phi"], fb["phi"])
            da, db = pg.pic_diagnostics(ens, k), pg.pic_diagnostics(one, 0)
            for key in ("N_e", "N_i", "V_cath", "I_cath", "n_sey", "n_ionize", "step"):
                assert da[key] == db[key], (k, key)
    stream.synchronize()


def test_ensemble_first_step_matches_oracle(pg):
    insts = _instances()
    ens = pg.pic_create([p for p, _ in insts])
    orcs = []
    for k, (p, parts) in enumerate(insts):
        _load(pg, ens, k, parts)
        orc = oracle.Oracle(p, parts)
        pg.pic_set_phi(ens, k, orc.fields()["phi"])
        orcs.append(orc)
    pg.pic_step(ens, 1)
    for k, orc in enumerate(orcs):
        orc.step(1)
        for sp in (0, 1):
            err = compare_species(pg.pic_get_particles(ens, k, sp), orc.get_particles(sp))
            assert err["pos"] <= PARTICLE_TOL and err["vel"] <= PARTICLE_TOL, (k, sp, err)


def test_ensemble_fp32_runs_and_tracks_fp64(pg):
    insts64 = _instances(0)
    insts32 = _instances(1)
    e64 = pg.pic_create([p for p, _ in insts64])
    e32 = pg.pic_create([p for p, _ in insts32])
    for k in range(len(insts64)):
        _load(pg, e64, k, insts64[k][1])
        _load(pg, e32, k, insts32[k][1])
        pg.pic_solve_fields(e64, k)
        pg.pic_solve_fields(e32, k)
    pg.pic_step(e64, 5)
    pg.pic_step(e32, 5)
    for k in range(len(insts64)):
        a, b = pg.pic_diagnostics(e32, k), pg.pic_diagnostics(e64, k)
        assert a["status"] == 0
        assert abs(a["N_e"] - b["N_e"]) <= max(2, 1e-4 * b["N_e"])
        assert a["W_field"] == pytest.approx(b["W_field"], rel=1e-3)


def test_mixed_grid_ensemble_equals_individual_runs(pg):
    """Instances of different grids (different multigrid hierarchies and
    single-CTA tails in the grouped Poisson launch) and particle counts."""
    insts = []
    for k, (nr, nz, ppc) in enumerate([(32, 48, 4), (64, 32, 6), (20, 36, 9)]):
        p = pic_inputs.params_rz32(gather=0)
        p.update(nr=nr, nz=nz, R=0.02, L=0.02 * nz / nr, Rc=0.6 * 0.02, gamma_i=0.2,
                 circuit_mode=1, Vs=400.0, Rext=100.0 * (k + 1), n_avg=4, seed=11 + k,
                 poisson_tol=1e-12)
        p, parts = busy_state(p, ppc=ppc, seed=200 + k)
        p = pic_inputs.with_capacity(p, parts, factor=2.0)
        insts.append((p, parts))
    steps = 6
    ens = pg.pic_create([p for p, _ in insts])
    for k, (p, parts) in enumerate(insts):
        _load(pg, ens, k, parts)
        pg.pic_solve_fields(ens, k)
    pg.pic_step(ens, steps)
    for k, (p, parts) in enumerate(insts):
        one = pg.pic_create(p)
        _load(pg, one, 0, parts)
        pg.pic_solve_fields(one, 0)
        pg.pic_step(one, steps)
        for sp in (0, 1):
            a = sort_by_id(pg.pic_get_particles(ens, k, sp))
            b = sort_by_id(pg.pic_get_particles(one, 0, sp))
            for q in a:
                assert np.array_equal(a[q], b[q]), (k, sp, q)
        assert np.array_equal(pg.pic_get_fields(ens, k)["phi"], pg.pic_get_fields(one, 0)["phi"])


def test_reweight_and_region_diagnostics_per_instance(pg):
    """Re-weighting one instance of an ensemble and sampling the region
    diagnostics of every instance give what the same discharges give one by
    one: particles, edges, cell counts and the ion histogram bit for bit; the
    temperatures to rounding (the velocity sums of a cell follow the order of
    its particles, which the cell sort does not fix)."""
    insts = _instances()
    for p, _ in insts:
        p.update(band_r_lo=0.006, band_r_hi=0.012, ied_bins=32, ied_emax=512.0)
    ens = pg.pic_create([p for p, _ in insts])
    for k, (p, parts) in enumerate(insts):
        _load(pg, ens, k, parts)
        pg.pic_solve_fields(ens, k)
    pg.pic_step(ens, 3)
    pg.pic_reweight(ens, 2, 3)
    for _ in range(3):
        pg.pic_step(ens, 1)
        for k in range(len(insts)):
            pg.pic_region_sample(ens, k)
    for k, (p, parts) in enumerate(insts):
        one = pg.pic_create(p)
        _load(pg, one, 0, parts)
        pg.pic_solve_fields(one, 0)
        pg.pic_step(one, 3)
        if k == 2:
            pg.pic_reweight(one, 0, 3)
        for _ in range(3):
            pg.pic_step(one, 1)
            pg.pic_region_sample(one, 0)
        for sp in (0, 1):
            a = sort_by_id(pg.pic_get_particles(ens, k, sp))
            b = sort_by_id(pg.pic_get_particles(one, 0, sp))
            for q in a:
                assert np.array_equal(a[q], b[q]), (k, sp, q)
        ra, rb = pg.pic_region_read(ens, k), pg.pic_region_read(one, 0)
        assert ra["samples"] == rb["samples"] == 3
        for key in ("ncell", "z_sheath", "z_bulk", "ion_impacts", "ied_overflow"):
            assert ra[key] == rb[key], (k, key)
        assert ra["Te"] == pytest.approx(rb["Te"], rel=1e-12), k
        for key in ("zs", "zb", "ied"):
            assert np.array_equal(ra[key], rb[key]), (k, key)
        assert pg.pic_diagnostics(ens, k)["weight"] == pg.pic_diagnostics(one, 0)["weight"]
        pg.pic_destroy(one)
    assert pg.pic_diagnostics(ens, 2)["weight"] == 3 * insts[2][0]["weight"]
    pg.pic_destroy(ens)


def test_periodic_sort_ensemble_equals_individual_runs(pg):
    """Full sorts every third step in an ensemble (each instance decides on
    its own state): still the single-instance results bit for bit."""
    import torch
    insts = _instances()
    for p, _ in insts:
        p["sort_every"] = 3
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ens = pg.pic_create([p for p, _ in insts])
        for k, (p, parts) in enumerate(insts):
            _load(pg, ens, k, parts)
            pg.pic_solve_fields(ens, k)
        pg.pic_step(ens, 8)
        for k, (p, parts) in enumerate(insts):
            one = pg.pic_create(p)
            _load(pg, one, 0, parts)
            pg.pic_solve_fields(one, 0)
            pg.pic_step(one, 8)
            assert pg.pic_diagnostics(ens, k)["N_e"] == pg.pic_diagnostics(one, 0)["N_e"]
            for sp in (0, 1):
                a = sort_by_id(pg.pic_get_particles(ens, k, sp))
                b = sort_by_id(pg.pic_get_particles(one, 0, sp))
                for q in a:
                    assert np.array_equal(a[q], b[q]), (k, sp, q)
            assert np.array_equal(pg.pic_get_fields(ens, k)["phi"], pg.pic_get_fields(one, 0)["phi"])
            pg.pic_destroy(one)
        pg.pic_destroy(ens)
    side.synchronize()


def test_autotuner_retunes_when_the_counts_grow(pg):
    """The push's chunk size and cell tile shape are tuned again when the live
    particle count has changed by a factor of 4 since the last tuning (an
    ensemble whose discharges grow); the tuning steps (the shape trials re-sort
    the particles) and the recaptured graph leave the results as they are: the
    ensemble still equals the instances run one by one, bit for bit, whatever
    shapes the ensemble and the single runs ended on."""
    import torch
    insts = []
    for k, (p, parts) in enumerate(_instances()):
        p = pic_inputs.with_capacity(p, parts, factor=16.0)
        insts.append((p, parts))
    grown = []
    for k, (p, _) in enumerate(insts):
        _, big = busy_state(dict(p), ppc=6 * (k + 4), seed=500 + k)
        grown.append(big)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        runs = [pg.pic_create([p for p, _ in insts])] + [pg.pic_create(p) for p, _ in insts]
        for k, (p, parts) in enumerate(insts):
            for h, j in ((runs[0], k), (runs[k + 1], 0)):
                _load(pg, h, j, parts)
                pg.pic_solve_fields(h, j)
        for h in runs:
            pg.pic_step(h, 6)      # four chunk sizes, two more tile shapes
        info0 = pg.pic_autotune_info(runs[0])
        assert info0["tunings"] == 1
        for k in range(len(insts)):
            for h, j in ((runs[0], k), (runs[k + 1], 0)):
                _load(pg, h, j, grown[k])
                pg.pic_solve_fields(h, j)
        for h in runs:
            pg.pic_step(h, 1)      # its end copies the grown count to the host
            pg.pic_sync(h)         # (the next call reads it once the copy is done)
            pg.pic_step(h, 6)      # sees it: six tuning steps, then the new graph
        info1 = pg.pic_autotune_info(runs[0])
        print("tunings", info0, info1, "tile shapes", [pg.pic_tuned_tile(h) for h in runs])
        assert info1["tunings"] == 2
        assert info1["particles_at_tuning"] >= 4 * info0["particles_at_tuning"]
        assert info1["particles_per_thread"] in (4, 8, 16, 32)
        pg.pic_step(runs[0], 3)
        assert pg.pic_uses_graph(runs[0])
        for k in range(len(insts)):
            pg.pic_step(runs[k + 1], 3)
            for sp in (0, 1):
                a = sort_by_id(pg.pic_get_particles(runs[0], k, sp))
                b = sort_by_id(pg.pic_get_particles(runs[k + 1], 0, sp))
                for q in a:
                    assert np.array_equal(a[q], b[q]), (k, sp, q)
        for h in runs:
            pg.pic_destroy(h)
    side.synchronize()
