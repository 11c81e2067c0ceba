"""The learned Poisson warm start on the GPU: network forward and gradients
against the FP64 reference network (oracle/unet.py), training on snapshots
the simulation records, and what the trained guess gains in the solve.

Tolerances (BF16 storage of activations and gradients, FP32 accumulation):
every activation and every gradient buffer is rounded to BF16 (relative
2^-9) once per layer; a CPU model of exactly these roundings gives a relative
L2 error of 4e-3 on the output, 1e-4 on the loss and up to 6e-2 on the
gradient of the first layer (the longest backward chain).  The bars below are
2.5-5x those figures; a dropped term, a wrong tap or a transposed operand
gives errors of order one.
"""
import numpy as np
import pytest
import torch

import pic_inputs
from oracle import unet
from parity import FIELD_TOL, field_err

pytestmark = pytest.mark.gpu

FWD_TOL = 2e-2
LOSS_TOL = 2e-3
GRAD_TOL = 0.15
GRAD_COS = 0.99


@pytest.fixture(scope="module")
def pg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2507_10727_gb300 as pg
    assert torch.cuda.is_available()
    return pg


def _bf16(a):
    return torch.tensor(a).to(torch.bfloat16).double().numpy()


def _oracle_params(seed):
    """He-normal weights, small random biases, rounded the way the GPU holds
    them: 3x3 weights in BF16, biases and the 1x1 head in FP32."""
    rng = np.random.default_rng(seed + 100)
    p = unet.init_params(seed)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.05 * rng.normal(size=p[k].shape)
        if k.endswith(".w") and not k.startswith("head"):
            p[k] = _bf16(p[k])
        else:
            p[k] = p[k].astype(np.float32).astype(np.float64)
    return p


def _flat(p):
    return np.concatenate([p[name + s].ravel() for name, _ in unet.layer_shapes()
                           for s in (".w", ".b")])


def _unflat(v):
    out, o = {}, 0
    for name, shp in unet.layer_shapes():
        n = int(np.prod(shp))
        out[name + ".w"] = v[o:o + n].reshape(shp)
        o += n
        out[name + ".b"] = v[o:o + shp[0]]
        o += shp[0]
    return out


def _handle(pg, nr=32, nz=64, batch=2):
    p = pic_inputs.params_rz32()
    p.update(nr=nr, nz=nz, L=p["R"] * nz / nr, cap_e=4096, cap_i=4096, birth_cap=1024)
    h = pg.pic_create(p)
    pg.pic_unet_create(h, 1, batch, 0)
    return h


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_forward_and_gradients_match_oracle(pg):
    h = _handle(pg)
    p = _oracle_params(7)
    flat = _flat(p)
    assert flat.size == pg.pic_unet_param_count()
    pg.pic_unet_set_params(h, flat)
    back = pg.pic_unet_get_params(h)
    assert np.array_equal(back, flat.astype(np.float32))
    rng = np.random.default_rng(3)
    x = _bf16(rng.normal(size=(2, 3, 33, 65)))
    y = rng.normal(size=(2, 1, 33, 65))
    out, g, loss = pg.pic_unet_loss_grad(h, x, y[:, 0])
    loss_o, g_o = unet.loss_and_grads(p, x, y)
    with torch.no_grad():
        out_o = unet.forward(p, torch.as_tensor(x)).numpy()[:, 0]
    assert _rel(out, out_o) <= FWD_TOL
    assert abs(loss - loss_o) <= LOSS_TOL * loss_o
    gg = _unflat(g.astype(np.float64))
    worst = 0.0
    for k in g_o:
        a, b = gg[k].ravel(), g_o[k].ravel()
        r = _rel(a, b)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        worst = max(worst, r)
        assert r <= GRAD_TOL and cos >= GRAD_COS, (k, r, cos)
    print(f"U-Net vs FP64 oracle: out {_rel(out, out_o):.2e}, loss {abs(loss - loss_o) / loss_o:.2e}, "
          f"worst gradient tensor {worst:.2e}")


def test_single_layer_paths_are_exact_in_structure(pg):
    """Identity-like weights (centre taps one on channel 0, the skip path of
    every decoder, head on channel 0): the output is x0 on every node, which
    pins the tap orientation, the even-node down-sampling, the concatenation
    order and the up-sampling of the CUDA path to the reference's."""
    h = _handle(pg, batch=1)
    p = unet.init_params(0)
    for k in p:
        p[k] = np.zeros_like(p[k])
    for name, shp in unet.layer_shapes():
        if shp[2] == 3:
            p[name + ".w"][0, 0, 1, 1] = 1.0
    for l in range(3):
        p[f"dec{l}a.w"][0, :, 1, 1] = 0.0
        p[f"dec{l}a.w"][0, unet.CHANNELS[l + 1], 1, 1] = 1.0
    p["head.w"][0, 0, 0, 0] = 1.0
    pg.pic_unet_set_params(h, _flat(p))
    rng = np.random.default_rng(5)
    x = _bf16(np.abs(rng.normal(size=(1, 3, 33, 65))))
    out, _, _ = pg.pic_unet_loss_grad(h, x)
    assert np.array_equal(out[0], x[0, 0].astype(np.float32))


def _simulation(pg, steps, mode, every=1, cap=128, seed=5, nr=32, nz=32, ppc=16, tol=1e-10):
    p = pic_inputs.params_rz32(gather=0)
    # the warm start serves the multigrid-preconditioned solve (with the
    # sine-transform preconditioner two iterations reach the tolerance from
    # any start)
    p.update(nr=nr, nz=nz, L=p["R"] * nz / nr, poisson_tol=tol, circuit_mode=1, Vs=400.0,
             Rext=500.0, n_avg=4, gamma_i=0.2, poisson_precond=1, poisson_max_iter=400)
    p, parts = pic_inputs.seed_plasma(p, nr * nz * ppc, seed=seed, Te_eV=5.0)
    p = pic_inputs.with_capacity(p, parts, factor=2.0)
    h = pg.pic_create(p)
    for k, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, 0, sp, parts[k])
    pg.pic_solve_fields(h, 0)
    pg.pic_unet_create(h, 2, 8, mode)
    pg.pic_unet_snapshots(h, cap, every)
    pg.pic_step(h, steps)
    pg.pic_sync(h)
    return p, h


def _iters(pg, h, steps):
    s0 = pg.pic_unet_stats(h)
    pg.pic_step(h, steps)
    s1 = pg.pic_unet_stats(h)
    return s1["poisson_iters"] - s0["poisson_iters"], {
        k: s1[k] - s0[k] for k in ("starts_previous", "starts_network", "starts_zero")}


@pytest.mark.parametrize("mode", [0, 1])
def test_training_reduces_the_loss(pg, mode):
    p, h = _simulation(pg, 48, mode)
    st = pg.pic_unet_stats(h)
    assert st["snapshots"] == 48
    first, last = pg.pic_unet_train(h, 300, 4, 2e-3, seed=1)
    st = pg.pic_unet_stats(h)
    assert st["in_norm"] > 0 and st["out_norm"] > 0
    assert np.isfinite(first) and np.isfinite(last)
    assert last < 0.2 * first, (first, last)


def _warm_and_plain(pg, mode, seed, tol, tmp_path, cold=False):
    """A run with a network trained on its own first 96 steps, checkpointed;
    the same state continued with the warm start on (the trained handle) and
    off (a fresh handle loaded from the checkpoint, whose network only counts
    iterations).  With `cold`, both solves of the next step start from phi = 0."""
    p, h = _simulation(pg, 96, mode, seed=seed, tol=tol)
    pg.pic_unet_train(h, 1500, 8, 2e-3, seed=seed)
    path = str(tmp_path / f"ck{mode}_{seed}.bin")
    pg.pic_save(h, 0, path)
    plain = pg.pic_create(p)
    pg.pic_load(plain, 0, path)
    pg.pic_unet_create(plain, 2, 1, mode)          # counts iterations; warm start off
    pg.pic_unet_warm_start(h, True)
    if cold:
        zero = np.zeros((p["nr"] + 1, p["nz"] + 1))
        pg.pic_set_phi(plain, 0, zero)
        pg.pic_set_phi(h, 0, zero)
    return p, h, plain


def test_correction_mode_saves_iterations(pg, tmp_path):
    """Mode 1 (the network predicts the change of phi from the residual of the
    previous solution): from identical states, 15 steps with the warm start
    need fewer multigrid-PCG iterations (to the library's 1e-10) than the
    plain solver started from the previous solution."""
    _, h, plain = _warm_and_plain(pg, 1, 9, 1e-10, tmp_path)
    off, _ = _iters(pg, plain, 15)
    on, starts = _iters(pg, h, 15)
    print(f"correction mode, 15 steps: Poisson iterations plain {off}, warm {on}; starts {starts}")
    assert starts["starts_network"] >= 8
    assert on < off


@pytest.mark.parametrize("mode, cold", [(1, False), (0, True)])
def test_warm_start_keeps_phi(pg, tmp_path, mode, cold):
    """The warm start changes where the solve starts, not what it reaches:
    with both arms solved to a 1e-13 relative residual (the condition number
    of the 32 x 32 operator is below 1e4) the next step's phi agree to 1e-10,
    for the correction mode from the previous solution and for the potential
    mode from a cold start (phi = 0)."""
    _, h, plain = _warm_and_plain(pg, mode, 21 + mode, 1e-13, tmp_path, cold=cold)
    off, _ = _iters(pg, plain, 1)
    on, starts = _iters(pg, h, 1)
    print(f"mode {mode}: Poisson iterations plain {off}, warm {on}; starts {starts}")
    assert starts["starts_network"] + starts["starts_previous"] + starts["starts_zero"] == 1
    assert field_err(pg.pic_get_fields(h, 0)["phi"], pg.pic_get_fields(plain, 0)["phi"]) <= \
        FIELD_TOL


def test_potential_mode_beats_a_cold_start(pg, tmp_path):
    """Mode 0 (the network maps rho, r and the electrode values to phi): a
    solve from phi = 0 (a cold start) needs fewer iterations with the warm
    start than without it."""
    _, h, plain = _warm_and_plain(pg, 0, 11, 1e-10, tmp_path, cold=True)
    off, _ = _iters(pg, plain, 1)
    on, starts = _iters(pg, h, 1)
    print(f"potential mode, cold start: Poisson iterations plain {off}, warm {on}; starts {starts}")
    assert starts["starts_network"] == 1
    assert on < off


def _sweep_instances(nr=32, nz=32, ppc=16):
    """Four discharges of the gamma x R_ext sweep on one 32 x 32 grid (the
    multigrid-preconditioned solve, as above)."""
    out = []
    for k, (gamma, rext) in enumerate([(0.05, 50.0), (0.1, 100.0), (0.2, 200.0), (0.3, 400.0)]):
        p = pic_inputs.params_rz32(gather=0)
        p.update(nr=nr, nz=nz, L=p["R"] * nz / nr, poisson_tol=1e-10, circuit_mode=1, Vs=400.0,
                 Rext=rext, n_avg=4, gamma_i=gamma, poisson_precond=1, poisson_max_iter=400,
                 seed=40 + k)
        p, parts = pic_inputs.seed_plasma(p, nr * nz * ppc, seed=50 + k, Te_eV=5.0)
        out.append((pic_inputs.with_capacity(p, parts, factor=2.0), parts))
    return out


def _begin(pg, h, k, parts):
    for key, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, k, sp, parts[key])
    pg.pic_solve_fields(h, k)


@pytest.mark.parametrize("mode", [0, 1])
def test_ensemble_network_equals_single_runs(pg, mode):
    """One network serves a 4-discharge ensemble.  Every instance records into
    the one ring (4 snapshots per step), training runs on the mixed ring, and
    the recording is then paused.
    With the warm start on, the batched forward (the 4 instances as one batch)
    gives each instance the start that a single-instance handle with the same
    network (parameters and scales) gives it: particles, phi, the step
    counters, the start choices and the iteration counts equal the single
    runs bit for bit, under graph replay."""
    from parity import sort_by_id
    insts = _sweep_instances()
    record_steps, steps = 24, 6
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ens = pg.pic_create([p for p, _ in insts])
        for k, (_, parts) in enumerate(insts):
            _begin(pg, ens, k, parts)
        pg.pic_unet_create(ens, 2, 8, mode)
        pg.pic_unet_snapshots(ens, 256, 1)
        pg.pic_step(ens, record_steps)
        assert pg.pic_unet_stats(ens)["snapshots"] == len(insts) * record_steps
        first, last = pg.pic_unet_train(ens, 300, 8, 2e-3, seed=3)
        assert last < first, (first, last)
        params = pg.pic_unet_get_params(ens)
        pg.pic_unet_record(ens, False)
        st = pg.pic_unet_stats(ens)
        pg.pic_unet_warm_start(ens, True)
        pg.pic_step(ens, steps)
        assert pg.pic_uses_graph(ens)
        s1 = pg.pic_unet_stats(ens)
        assert s1["snapshots"] == st["snapshots"]   # recording paused
        totals = {"starts_previous": 0, "starts_network": 0, "starts_zero": 0,
                  "poisson_iters": 0}
        for k, (p, parts) in enumerate(insts):
            one = pg.pic_create(p)
            _begin(pg, one, 0, parts)
            pg.pic_step(one, record_steps)   # the state of instance k (FP64: bit for bit)
            pg.pic_unet_create(one, 2, 1, mode)
            pg.pic_unet_set_params(one, params)
            pg.pic_unet_set_norms(one, st["in_norm"], st["out_norm"])
            pg.pic_unet_warm_start(one, True)
            pg.pic_step(one, steps)
            so = pg.pic_unet_stats(one)
            for key in totals:
                totals[key] += so[key]
            for sp in (0, 1):
                a = sort_by_id(pg.pic_get_particles(ens, k, sp))
                b = sort_by_id(pg.pic_get_particles(one, 0, sp))
                for q in a:
                    assert np.array_equal(a[q], b[q]), (k, sp, q)
            assert np.array_equal(pg.pic_get_fields(ens, k)["phi"],
                                  pg.pic_get_fields(one, 0)["phi"]), k
            da, db = pg.pic_diagnostics(ens, k), pg.pic_diagnostics(one, 0)
            for key in ("N_e", "N_i", "V_cath", "I_cath", "step", "poisson_iters"):
                assert da[key] == db[key], (k, key)
            pg.pic_destroy(one)
        print(f"mode {mode}: ensemble starts/iterations over {steps} steps:",
              {key: s1[key] - st[key] for key in totals})
        for key in totals:
            assert s1[key] - st[key] == totals[key], key
        pg.pic_destroy(ens)
    side.synchronize()
