"""Seeded synthetic inputs for the RZ PIC-MCC discharge: run parameters and initial plasmas.

This module is shared by the CUDA library's tests and benchmark and by the CPU
oracle's tests. It holds no step of the method: no push, gather, deposit,
collision or field-solve arithmetic. It only produces

* run-parameter dictionaries (plain numbers) for the workloads named below, and
* initial particle populations drawn with numpy's seeded generators.

Workloads (all synthetic; the paper's VSim inputs -- QDB cross sections, the
magnet's field, the 3 x 3 cm geometry -- are not available, so analytic
stand-ins are used, see the per-function docstrings):

* ``rz32``        32 x 32 cells, R = L = 2.5 cm, cathode fixed at -400 V, 64
                  macroparticles per cell per species (65,536 each), dt = 50 ps.
* ``rz256``       256 x 256 cells, R = L = 5 cm, external circuit V_s = 500 V,
                  R_ext = 200 Ohm, dt = 30 ps; loaded either as the uniform
                  1e15 m^-3 seed plasma or as a "grown" state with a Gaussian
                  racetrack ring near the cathode (Section 4 describes the
                  plasma localised next to the cathode).
* ``rz128_sweep`` 16 discharges on 128 x 128 cells, gamma x R_ext sweep.
* ``rz256x512``   256 x 512 cells, R = 5 cm, L = 10 cm.

The key names of the parameter dictionaries are the field names of the C
structs of both the CUDA library (``include/pic.h``) and the oracle.
"""
from __future__ import annotations

import math

import numpy as np

# CODATA 2018 values.
E_CHARGE = 1.602176634e-19      # C
M_ELECTRON = 9.1093837015e-31   # kg
AMU = 1.66053906660e-27         # kg
M_ARGON = 39.948 * AMU          # kg
EPS0 = 8.8541878128e-12         # F/m
K_BOLTZMANN = 1.380649e-23      # J/K
TORR = 133.322368421            # Pa

# Species tags (also the Philox key's second word).
ELECTRON = 0
ION = 1


def gas_density(p_mtorr: float, T_gas: float) -> float:
    """Ideal-gas number density (m^-3) of the background argon."""
    return p_mtorr * 1e-3 * TORR / (K_BOLTZMANN * T_gas)


def base_params() -> dict:
    """Parameters common to every workload (Section 3 and the analytic stand-ins).

    Cross-section stand-ins: elastic 1e-19 m^2 (constant); excitation with
    threshold 11.55 eV (reaction 1b) and ionization with threshold 15.76 eV
    (reaction 1c) of the Lotz single-shell form; stepwise ionization from the
    metastable Ar* (reaction 1d, threshold 4.20 eV, one outer electron) off a
    constant Ar* background of density n_meta (0 unless a workload sets it;
    the paper's runs use 2.5e17 m^-3).  The magnetron field is the
    vacuum field B = -grad(A0 J0(kr) exp(-kz)) with k = 3.83 / 2 cm and
    k A0 = 0.04 T, so that B_r vanishes at the cathode edge r = 2 cm.
    """
    return dict(
        nr=32, nz=32, R=0.025, L=0.025, Rc=0.02,
        dt=5e-11, weight=1.0,
        m_ion=M_ARGON, n_gas=gas_density(3.0, 300.0), T_gas=300.0,
        b_mode=0, B_kA0=0.04, B_k=3.83 / 0.02, B0r=0.0, B0z=0.0,
        gamma_i=0.1, gamma_e=0.0,
        circuit_mode=0, Vc_fixed=-400.0, Vs=400.0, Rext=0.0, n_avg=100,
        gather=0, rweight=0, precision=0,
        mcc_on=1, push_on=1, field_on=1, walls_reflect=0,
        seed=0,
        sigma_el=1e-19, ion_a=4.0e-18 * 6.0, ion_I=15.76,
        exc_C=3.63e-18, exc_E=11.55, E_cap=800.0,
        n_meta=0.0, meta_a=4.0e-18, meta_I=4.20,
        gap_neumann=0, wall_neumann=0,
        band_r_lo=0.010, band_r_hi=0.015, ied_bins=0, ied_emax=600.0,
        poisson_tol=1e-10, poisson_max_iter=200, phi_extrapolate=0, poisson_precond=0,
        cap_e=0, cap_i=0, birth_cap=0, diag_every=1,
        sort_every=1,
    )


def params_rz32(gather: int = 0, precision: int = 0, seed: int = 0) -> dict:
    """32 x 32 RZ cylinder, cathode disk r <= 2 cm fixed at -400 V, 500 steps of 50 ps."""
    p = base_params()
    p.update(nr=32, nz=32, R=0.025, L=0.025, Rc=0.02, dt=5e-11,
             circuit_mode=0, Vc_fixed=-400.0, Vs=400.0, E_cap=800.0,
             gather=gather, precision=precision, seed=seed)
    return p


def params_rz256(gather: int = 0, precision: int = 0, seed: int = 0) -> dict:
    """256 x 256 cells over 5 cm x 5 cm, external circuit V_s = 500 V, R_ext = 200 Ohm."""
    p = base_params()
    p.update(nr=256, nz=256, R=0.05, L=0.05, Rc=0.02, dt=3e-11,
             circuit_mode=1, Vc_fixed=-500.0, Vs=500.0, Rext=200.0, n_avg=100,
             E_cap=1000.0, gather=gather, precision=precision, seed=seed)
    return p


def params_rz256x512(gather: int = 0, precision: int = 0, seed: int = 0) -> dict:
    """256 (r) x 512 (z) cells over R = 5 cm, L = 10 cm."""
    p = params_rz256(gather, precision, seed)
    p.update(nr=256, nz=512, R=0.05, L=0.10)
    return p


def params_paper(gather: int = 0, precision: int = 0, seed: int = 0, cells: int = 256,
                 gamma_i: float = 0.1, Rext: float = 3000.0) -> dict:
    """The paper's chamber (Section 3): 3 cm x 3 cm, cathode r <= 0.85 L_r on
    z = 0, the rest of z = 0 the insulating block (Neumann), anode z = L and
    wall r = R grounded, 10 mTorr, V_ext = -300 V through R_ext (3000 or
    1000 Ohm), ion SEY 0.1 / 0.2, electron SEY 0.1, Ar* background
    2.5e17 m^-3.  The magnet field stand-in puts the racetrack (B_z = 0) at
    r = 1.2 cm (k r = 2.405), between the paper's inner magnet (6.5 mm) and
    outer magnet (1.7 cm).  `cells` x `cells` grid; 20 ps steps."""
    p = base_params()
    p.update(nr=cells, nz=cells, R=0.03, L=0.03, Rc=0.85 * 0.03, dt=2e-11,
             n_gas=gas_density(10.0, 300.0), gap_neumann=1, wall_neumann=0,
             circuit_mode=1, Vc_fixed=-300.0, Vs=300.0, Rext=Rext, n_avg=100,
             gamma_i=gamma_i, gamma_e=0.1, n_meta=2.5e17, B_k=2.405 / 0.012,
             E_cap=600.0, ied_bins=160, ied_emax=320.0,
             gather=gather, precision=precision, seed=seed)
    return p


# Long-run statistics of the 32 x 32 discharge with the external circuit
# ("cfg 1L": V_s = 400 V, R_ext = 200 Ohm, 1e5 steps of 50 ps = 5 us): the
# averages are taken over the second half, sampled every STEADY_EVERY steps.
STEADY_STEPS = 100_000
STEADY_WINDOW = 50_000
STEADY_EVERY = 50


def steady_cfg1L(seed: int, gather: int = 0, precision: int = 0) -> tuple[dict, dict]:
    """The 32 x 32 discharge of ``params_rz32`` with the external circuit
    V_s = 400 V, R_ext = 200 Ohm (100-step current average), seeded by
    ``seed`` (Philox key and the seed plasma's draw): 64 macroparticles per
    cell per species of a uniform 1e15 m^-3, 2 eV / 0.026 eV plasma."""
    p = params_rz32(gather=gather, precision=precision, seed=seed)
    p.update(circuit_mode=1, Vs=400.0, Rext=200.0, n_avg=100, diag_every=STEADY_EVERY,
             poisson_tol=1e-10)
    p, parts = seed_plasma(p, 32 * 32 * 64, n0=1e15, seed=1000 + seed)
    return with_capacity(p, parts, factor=2.0, births=1 << 16), parts


def params_rz128_sweep(gather: int = 0, precision: int = 0, seed: int = 0) -> list[dict]:
    """16 independent 128 x 128 discharges: gamma in {.05,.1,.2,.3} x R_ext in {50,100,200,400} Ohm."""
    out = []
    for gamma in (0.05, 0.1, 0.2, 0.3):
        for rext in (50.0, 100.0, 200.0, 400.0):
            p = params_rz256(gather, precision, seed)
            p.update(nr=128, nz=128, gamma_i=gamma, Rext=rext, seed=seed + len(out))
            out.append(p)
    return out


def _maxwellian(rng: np.random.Generator, n: int, T_eV: float, mass: float) -> np.ndarray:
    sigma = math.sqrt(T_eV * E_CHARGE / mass)
    return rng.normal(0.0, sigma, size=(3, n))


def _assemble(r, z, ve, vi, id0: int = 0) -> dict:
    n = r.shape[0]
    e = dict(r=r.copy(), z=z.copy(), vr=ve[0].copy(), vt=ve[1].copy(), vz=ve[2].copy(),
             id=np.arange(id0, id0 + n, dtype=np.int64))
    i = dict(r=r.copy(), z=z.copy(), vr=vi[0].copy(), vt=vi[1].copy(), vz=vi[2].copy(),
             id=np.arange(id0 + n, id0 + 2 * n, dtype=np.int64))
    return {"e": e, "i": i}


def seed_plasma(params: dict, n_per_species: int, n0: float = 1e15, Te_eV: float = 2.0,
                Ti_eV: float = 0.026, seed: int = 0) -> tuple[dict, dict]:
    """Uniform-density seed plasma (Section 4: "seed population of uniform density").

    Positions are uniform in volume (r = R sqrt(U), z = L U); electrons and ions
    share positions so the initial charge density is zero up to shape
    differences; velocities are Maxwellian (T_e, T_i).  Returns the updated
    parameters (weight set so that the density is ``n0``) and the particles.
    Electron ids are 0..N-1, ion ids N..2N-1.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    R, L = params["R"], params["L"]
    n = int(n_per_species)
    r = R * np.sqrt(rng.random(n))
    z = L * rng.random(n)
    ve = _maxwellian(rng, n, Te_eV, M_ELECTRON)
    vi = _maxwellian(rng, n, Ti_eV, params["m_ion"])
    p = dict(params)
    p["weight"] = n0 * math.pi * R * R * L / max(n, 1)
    return p, _assemble(r, z, ve, vi)


def grown_ring_state(params: dict, n_per_species: int, n_floor: float = 1e15,
                     n_ring: float = 1e16, r0: float = 0.0125, z0: float = 0.002,
                     sig_r: float = 0.003, sig_z: float = 0.002, Te_eV: float = 2.0,
                     Ti_eV: float = 0.026, seed: int = 0) -> tuple[dict, dict]:
    """Synthetic developed discharge: uniform floor plus a Gaussian racetrack ring.

    Density n(r,z) = n_floor + n_ring exp(-(r-r0)^2/2 sig_r^2 - (z-z0)^2/2 sig_z^2),
    the cathode-localised plasma of Section 4 (peak near the cathode sheath, at
    r ~ 1.25 cm here).  Particles are drawn from n(r,z) 2 pi r dr dz by mixture
    sampling; the macroparticle weight follows from the total real count.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    R, L = params["R"], params["L"]
    n = int(n_per_species)
    # Real-particle content of the two mixture parts (ring part by quadrature).
    floor_count = n_floor * math.pi * R * R * L
    rr = (np.arange(4096) + 0.5) * (R / 4096)
    zz = (np.arange(4096) + 0.5) * (L / 4096)
    gr = np.exp(-(rr - r0) ** 2 / (2 * sig_r ** 2)) * 2 * math.pi * rr
    gz = np.exp(-(zz - z0) ** 2 / (2 * sig_z ** 2))
    ring_count = n_ring * gr.sum() * (R / 4096) * gz.sum() * (L / 4096)
    total = floor_count + ring_count
    n_ring_part = int(round(n * ring_count / total))
    n_floor_part = n - n_ring_part
    r = np.empty(n)
    z = np.empty(n)
    r[:n_floor_part] = R * np.sqrt(rng.random(n_floor_part))
    z[:n_floor_part] = L * rng.random(n_floor_part)
    filled = 0
    while filled < n_ring_part:
        m = max(1024, int(1.5 * (n_ring_part - filled)))
        rc = rng.normal(r0, sig_r, m)
        zc = rng.normal(z0, sig_z, m)
        acc = (rc > 0) & (rc < R) & (zc >= 0) & (zc < L) & (rng.random(m) * R < rc)
        rc, zc = rc[acc], zc[acc]
        k = min(rc.shape[0], n_ring_part - filled)
        r[n_floor_part + filled:n_floor_part + filled + k] = rc[:k]
        z[n_floor_part + filled:n_floor_part + filled + k] = zc[:k]
        filled += k
    perm = rng.permutation(n)
    r, z = r[perm], z[perm]
    ve = _maxwellian(rng, n, Te_eV, M_ELECTRON)
    vi = _maxwellian(rng, n, Ti_eV, params["m_ion"])
    p = dict(params)
    p["weight"] = total / max(n, 1)
    return p, _assemble(r, z, ve, vi)


def with_capacity(params: dict, particles: dict, factor: float = 1.5, births: int = 0) -> dict:
    """Return parameters with particle capacities sized for growth by ``factor``."""
    p = dict(params)
    ne = particles["e"]["r"].shape[0]
    ni = particles["i"]["r"].shape[0]
    p["cap_e"] = max(1024, int(factor * ne))
    p["cap_i"] = max(1024, int(factor * ni))
    p["birth_cap"] = births if births else max(4096, (ne + ni) // 64)
    return p
