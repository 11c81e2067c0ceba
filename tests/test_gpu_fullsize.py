"""Parity at the sizes the benchmark runs, element by element against the
oracle (Sections 2-3: deposit and gather, walls, MCC; the step order of the
oracle).

The small-grid tests of test_gpu_parity.py never reach the paths the kernels
take on the benchmark's workloads; these do:

* the 256 x 256 cell chamber (5 cm x 5 cm, external circuit) in the synthetic
  grown-ring state, 2e6 macroparticles per species, the push fixed at 32
  particles per thread (8192-particle chunks, more chunks than persistent
  CTAs), the cell sort every 32 steps and the steps on both sides of one (the
  in-place steps append births and keep dead slots; the sparse floor region
  makes chunks span many tiles, so the deposit patch spills to global atomics),
  the extrapolated Poisson start -- FP64 EC and MC at 1e-12, FP32 at 1e-5;
* the 16-instance 128 x 128 gamma x R_ext sweep with uneven counts
  (2e4 - 2e5 per species, and the benchmark's 1e6 - 8e6) under CUDA-graph
  replay;
* one step on the 256 x 512 grid of the learned warm-start workload;
* the benchmark's own size, 4e7 per species on 256 x 256, in its launch
  configuration (32 particles per thread, 8 x 8 tiles), FP64 and FP32, the
  full-sort step and the one after it.
"""
import math

import numpy as np
import pytest

import oracle
import pic_inputs
from parity import check_step64, field_err

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def pg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_10727_gb300 as pg
    import torch
    assert torch.cuda.is_available()
    return pg


def _ring(p, n, seed):
    p, parts = pic_inputs.grown_ring_state(p, n, seed=seed)
    return pic_inputs.with_capacity(p, parts, factor=1.5), parts


def _start(pg, h, orc, parts, k=0, step=30):
    """Load the oracle's state into instance k and put both sides at step
    index `step` (the full sort ends step 31 of every 32)."""
    for key, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, k, sp, parts[key])
    pg.pic_set_phi(h, k, orc.fields()["phi"])
    V0 = -orc.p["Vs"]
    qh = np.zeros(orc.p["n_avg"])
    orc.set_circuit(V0, step, qh)
    pg.pic_set_circuit(h, k, V0, step, qh)


@pytest.mark.parametrize("gather", [0, 1])
def test_rz256_ring_fp64_steps_around_a_full_sort(pg, gather):
    p = pic_inputs.params_rz256(gather=gather)
    p.update(poisson_tol=1e-13, sort_every=32, phi_extrapolate=1)
    p, parts = _ring(p, 2_000_000, seed=5 + gather)
    orc = oracle.Oracle(p, parts)
    h = pg.pic_create(p)
    _start(pg, h, orc, parts)
    pg.pic_set_chunk(h, 32)
    for step in (30, 31, 32):   # in place, ends with the full sort, in place
        orc.step(1)
        pg.pic_step(h, 1)
        d = check_step64(pg, h, orc)
        assert d["step"] == step
        assert pg.pic_tuned_chunk(h) == 32
    # the steps do meet the cathode (electrons; the 0.026 eV ions of the ring
    # move a few tens of nanometres in three steps) and collide
    assert d["n_e_cath"] > 0 and d["n_ionize"] + d["n_excite"] + d["n_elastic"] > 0
    assert pg.pic_get_next_id(h, 0) == orc.next_id
    pg.pic_destroy(h)


def _compare32(a, b):
    """FP32 particles `a` against FP64 oracle particles `b`: relative errors
    over the particles that took the same discrete decisions, and the number
    that did not (different id sets, or a velocity that misses the FP32 bar: a
    different collision branch or scattering reference axis; see
    test_gpu_fp32)."""
    ia, ib = np.sort(a["id"]), np.sort(b["id"])
    common = np.intersect1d(ia, ib, assume_unique=True)
    flips = int(ia.size + ib.size - 2 * common.size)
    oa, ob = np.argsort(a["id"]), np.argsort(b["id"])
    sa = oa[np.isin(a["id"][oa], common)]
    sb = ob[np.isin(b["id"][ob], common)]
    va = np.stack([a["vr"][sa], a["vt"][sa], a["vz"][sa]])
    vb = np.stack([b["vr"][sb], b["vt"][sb], b["vz"][sb]])
    vmax = max(np.abs(vb).max(), 1e-300) if vb.size else 1.0
    branch = np.abs(va - vb).max(axis=0) > TOL32 * vmax
    flips += int(branch.sum())
    keep = ~branch
    pa = np.stack([a["r"][sa], a["z"][sa]])[:, keep]
    pb = np.stack([b["r"][sb], b["z"][sb]])[:, keep]
    return (float(np.abs(pa - pb).max() / np.abs(pb).max()),
            float(np.abs(va[:, keep] - vb[:, keep]).max() / vmax), flips)


def test_rz256_ring_fp32_steps_around_a_full_sort(pg):
    p = pic_inputs.params_rz256(gather=0)
    p.update(poisson_tol=1e-12, sort_every=32, phi_extrapolate=1)
    p, parts = _ring(p, 2_000_000, seed=9)
    orc = oracle.Oracle(p, parts)
    h = pg.pic_create(dict(p, precision=1))
    _start(pg, h, orc, parts)
    pg.pic_set_chunk(h, 32)
    for _ in range(3):
        orc.step(1)
        pg.pic_step(h, 1)
        n_total, flips = 0, 0
        for sp in (0, 1):
            b = orc.get_particles(sp)
            pos, vel, f = _compare32(pg.pic_get_particles(h, 0, sp), b)
            assert pos <= TOL32 and vel <= TOL32, (sp, pos, vel)
            n_total += b["id"].size
            flips += f
        assert flips <= math.ceil(1e-5 * n_total), flips
        # the deposit (each species' node charge) and the field at the FP32 bar;
        # the net charge is their difference, nearly cancelling in this
        # quasi-neutral state, so its error relative to its own (small)
        # maximum is not bounded separately
        for sp in (0, 1):
            err = field_err(pg.pic_get_species_charge(h, 0, sp), orc.species_charge(sp))
            assert err <= TOL32, (sp, err)
        fg, fo = pg.pic_get_fields(h, 0), orc.fields()
        assert field_err(fg["phi"], fo["phi"]) <= TOL32
    pg.pic_destroy(h)


@pytest.fixture(scope="module")
def bench_state():
    """The benchmark's workload: the 256 x 256 grown-ring state with 4e7
    macroparticles per species (bench.py's default size)."""
    p = pic_inputs.params_rz256(gather=0)
    p.update(poisson_tol=1e-13, sort_every=32, phi_extrapolate=1)
    return _ring(p, 40_000_000, seed=0)


@pytest.mark.parametrize("precision", [0, 1])
def test_bench_size_steps_around_a_full_sort(pg, bench_state, precision):
    """The benchmark's size and launch configuration: 4e7 macroparticles per
    species on 256 x 256 cells, the push at 32 particles per thread on 8 x 8
    cell tiles (what the autotuner takes at this size), the step that ends with
    the full sort and the in-place step after it; every particle, the node
    charges and the field against the oracle (FP64 at 1e-12, the FP32 mode at
    1e-5 with its flip budget)."""
    p, parts = bench_state
    orc = oracle.Oracle(p, parts)
    h = pg.pic_create(dict(p, precision=precision))
    _start(pg, h, orc, parts, step=31)
    pg.pic_set_chunk(h, 32)
    pg.pic_set_tile(h, 1)
    for step in (31, 32):   # ends with the full sort, then in place
        orc.step(1)
        pg.pic_step(h, 1)
        assert pg.pic_tuned_chunk(h) == 32 and pg.pic_tuned_tile(h) == 1
        if precision == 0:
            d = check_step64(pg, h, orc)
            assert d["step"] == step
            continue
        n_total, flips = 0, 0
        for sp in (0, 1):
            b = orc.get_particles(sp)
            pos, vel, f = _compare32(pg.pic_get_particles(h, 0, sp), b)
            assert pos <= TOL32 and vel <= TOL32, (sp, pos, vel)
            n_total += b["id"].size
            flips += f
            err = field_err(pg.pic_get_species_charge(h, 0, sp), orc.species_charge(sp))
            assert err <= TOL32, (sp, err)
        assert flips <= math.ceil(1e-5 * n_total), flips
        assert field_err(pg.pic_get_fields(h, 0)["phi"], orc.fields()["phi"]) <= TOL32
    d = pg.pic_diagnostics(h, 0)
    assert d["n_e_cath"] > 0 and d["n_ionize"] > 0
    pg.pic_destroy(h)
    del orc


def test_sweep16_ensemble_uneven_counts_graph_replay(pg):
    """16 discharges of 128 x 128 cells (gamma x R_ext sweep) in one handle,
    2e4 .. 2e5 macroparticles per species spread unevenly over the instances,
    stepped by replaying the captured step graph on a side stream; every
    instance matches its own oracle after each step."""
    import torch
    plist = pic_inputs.params_rz128_sweep()
    order = np.random.default_rng(4).permutation(16)
    insts = []
    for k, p in enumerate(plist):
        n = int(round(2e4 * 10.0 ** (order[k] / 15.0)))
        p.update(poisson_tol=1e-13, sort_every=32)
        insts.append(_ring(p, n, seed=300 + k))
    orcs = [oracle.Oracle(p, parts) for p, parts in insts]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        h = pg.pic_create([p for p, _ in insts])
        for k, ((p, parts), orc) in enumerate(zip(insts, orcs)):
            _start(pg, h, orc, parts, k=k)
        pg.pic_set_chunk(h, 32)
        for _ in range(2):   # step 30 in place, step 31 ends with the full sort
            pg.pic_step(h, 1)
            assert pg.pic_uses_graph(h)
            for k, orc in enumerate(orcs):
                orc.step(1)
                check_step64(pg, h, orc, instance=k)
        pg.pic_destroy(h)
    side.synchronize()


def test_sweep16_ensemble_bench_sizes(pg):
    """The sweep at the benchmark's sizes: 16 discharges of 128 x 128 cells with
    1e6 8^(k/15) macroparticles per species (1e6 .. 8e6, 1.1e8 in all, shuffled
    over the gamma x R_ext grid), the push at 32 particles per thread, stepped
    by graph replay through the step that ends with the full sort and the one
    after it; every instance against its own oracle after each step."""
    import torch
    plist = pic_inputs.params_rz128_sweep()
    sizes = [int(1e6 * 8.0 ** (k / 15.0)) for k in range(16)]
    np.random.default_rng(5).shuffle(sizes)
    insts = []
    for k, p in enumerate(plist):
        p.update(poisson_tol=1e-13, sort_every=32, phi_extrapolate=1)
        insts.append(_ring(p, sizes[k], seed=31 * k))
    orcs = [oracle.Oracle(p, parts) for p, parts in insts]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        h = pg.pic_create([p for p, _ in insts])
        for k, ((p, parts), orc) in enumerate(zip(insts, orcs)):
            _start(pg, h, orc, parts, k=k, step=31)
        pg.pic_set_chunk(h, 32)
        for step in (31, 32):   # ends with the full sort, then in place
            pg.pic_step(h, 1)
            assert pg.pic_uses_graph(h)
            for k, orc in enumerate(orcs):
                orc.step(1)
                d = check_step64(pg, h, orc, instance=k)
                assert d["step"] == step
        pg.pic_destroy(h)
    side.synchronize()


def test_rz256x512_one_step(pg):
    p = pic_inputs.params_rz256x512(gather=0)
    p.update(poisson_tol=1e-13)
    p, parts = _ring(p, 1_000_000, seed=13)
    orc = oracle.Oracle(p, parts)
    h = pg.pic_create(p)
    _start(pg, h, orc, parts, step=0)
    orc.step(1)
    pg.pic_step(h, 1)
    check_step64(pg, h, orc)
    pg.pic_destroy(h)


def _one_cell(p, n, seed=0):
    """n electrons and n ions in one cell (10, 10) of the 32 x 32 grid."""
    rng = np.random.default_rng(seed)
    dr, dz = p["R"] / p["nr"], p["L"] / p["nz"]
    r = (10 + rng.random(n)) * dr
    z = (10 + rng.random(n)) * dz
    v = np.zeros(n)
    e = dict(r=r, z=z, vr=v, vt=v, vz=v, id=np.arange(n, dtype=np.int64))
    i = dict(r=r, z=z, vr=v, vt=v, vz=v, id=np.arange(n, 2 * n, dtype=np.int64))
    return {"e": e, "i": i}


def test_fixed_point_deposit_capacity_guard(pg):
    """FP64 node charges are 44-bit fixed-point sums in 64-bit words, so a
    node holds fewer than 2^20 macroparticles; a node gathers from four cells,
    so a cell with 2^18 macroparticles of one species latches
    PIC_ERR_CAPACITY (at its sort) instead of letting a sum wrap.  One fewer
    is accepted; FP32 particles (FP64 node sums) have no such bound."""
    from paper_2507_10727_gb300.pic import PicError
    p = pic_inputs.params_rz32()
    p.update(mcc_on=0, push_on=0)
    for n, precision, ok in ((1 << 18, 0, False), ((1 << 18) - 1, 0, True), (1 << 18, 1, True)):
        parts = _one_cell(p, n)
        q = pic_inputs.with_capacity(dict(p, precision=precision), parts, factor=1.1)
        h = pg.pic_create(q)
        if ok:
            for key, sp in (("e", 0), ("i", 1)):
                pg.pic_set_particles(h, 0, sp, parts[key])
            pg.pic_step(h, 1)
            d = pg.pic_diagnostics(h, 0)
            assert d["ppc_max_e"] == n and d["ppc_max_i"] == n
            # push off: every particle stays; the species charges are exact
            Qe = pg.pic_get_species_charge(h, 0, 0)
            assert Qe.sum() == pytest.approx(-n * pic_inputs.E_CHARGE * q["weight"], rel=1e-12)
        else:
            with pytest.raises(PicError) as err:
                pg.pic_set_particles(h, 0, 0, parts["e"])
            assert err.value.code == -3
        pg.pic_destroy(h)
