"""Write tests/golden/steady_cfg1L.txt: long-run statistics of the 32 x 32
discharge with the external circuit (pic_inputs.steady_cfg1L), computed by the
CPU oracle alone, one seed per process.

For every seed s = 0 .. 63: the run of pic_inputs.STEADY_STEPS steps, sampled
every STEADY_EVERY steps over the last STEADY_WINDOW of them (Section 4 takes
its steady-state values as time averages); the columns are the averages of
the cathode current I (A), the cathode potential V_c (V), the macroparticle
counts N_e, N_i, and each species' peak density (m^-3): the largest
time-averaged density of a neighbourhood of PEAK_NODES x PEAK_NODES nodes
(clipped at the walls), i.e. the neighbourhood's deposited charge over its
volume, a node's volume being the part of the cylinder within half a cell of
the node.  At the ten or so macroparticles per cell of this state the density
of a single node -- an axis node's volume pi (dr/2)^2 dz holds less than one
macroparticle -- is sampling noise; at the 7 x 7 node (5.5 mm) scale the
seed-to-seed spread of the peak is about 6 %, so the mean of 64 seeds is
known to about 0.7 %.  The last two columns give the single-node peaks for
information.

Run from the repository root:  python tests/golden/make_steady_state.py
(about 75 minutes on eight cores).
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import pic_inputs  # noqa: E402

SEEDS = range(64)
PEAK_NODES = 7
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "steady_cfg1L.txt")


def neighbourhood_peak(q: np.ndarray, vol: np.ndarray, w: int) -> float:
    """Largest (sum of q) / (sum of vol) over the w x w node neighbourhoods
    centred on the nodes (clipped at the grid's edges)."""
    h = w // 2
    best = 0.0
    for m in range(q.shape[0]):
        for n in range(q.shape[1]):
            sl = (slice(max(0, m - h), m + h + 1), slice(max(0, n - h), n + h + 1))
            best = max(best, float(q[sl].sum() / vol[sl].sum()))
    return best


def control_volumes(p: dict) -> np.ndarray:
    dr, dz = p["R"] / p["nr"], p["L"] / p["nz"]
    m = np.arange(p["nr"] + 1)[:, None]
    n = np.arange(p["nz"] + 1)[None, :]
    r_lo, r_hi = np.maximum(0.0, (m - 0.5) * dr), np.minimum(p["R"], (m + 0.5) * dr)
    z_lo, z_hi = np.maximum(0.0, (n - 0.5) * dz), np.minimum(p["L"], (n + 0.5) * dz)
    return math.pi * (r_hi ** 2 - r_lo ** 2) * (z_hi - z_lo)


def run_seed(seed: int) -> list[float]:
    import oracle
    p, parts = pic_inputs.steady_cfg1L(seed)
    orc = oracle.Oracle(p, parts)
    first = pic_inputs.STEADY_STEPS - pic_inputs.STEADY_WINDOW
    orc.step(first)
    every = pic_inputs.STEADY_EVERY
    acc = {"I": 0.0, "V": 0.0, "Ne": 0.0, "Ni": 0.0}
    qe = np.zeros((p["nr"] + 1, p["nz"] + 1))
    qi = np.zeros_like(qe)
    k = 0
    for _ in range(pic_inputs.STEADY_WINDOW // every):
        orc.step(every)
        d = orc.diag()
        acc["I"] += d["I_cath"]
        acc["V"] += d["V_cath"]
        acc["Ne"] += d["N_e"]
        acc["Ni"] += d["N_i"]
        qe += orc.species_charge(0)
        qi += orc.species_charge(1)
        k += 1
    vol = control_volumes(p)
    ne = np.abs(qe) / k / pic_inputs.E_CHARGE      # time-averaged macroparticle charge / e
    ni = np.abs(qi) / k / pic_inputs.E_CHARGE
    return [seed, acc["I"] / k, acc["V"] / k, acc["Ne"] / k, acc["Ni"] / k,
            neighbourhood_peak(ne, vol, PEAK_NODES), neighbourhood_peak(ni, vol, PEAK_NODES),
            (ne / vol).max(), (ni / vol).max()]


def main():
    from oracle import build
    build.build()
    with mp.get_context("spawn").Pool(min(len(SEEDS), os.cpu_count() or 1)) as pool:
        rows = pool.map(run_seed, list(SEEDS))
    with open(OUT, "w") as f:
        f.write("# Long-run statistics of the 32x32 discharge with the external circuit\n")
        f.write("# (pic_inputs.steady_cfg1L: V_s = 400 V, R_ext = 200 Ohm), CPU oracle;\n")
        f.write(f"# {pic_inputs.STEADY_STEPS} steps, averages over the last "
                f"{pic_inputs.STEADY_WINDOW} sampled every {pic_inputs.STEADY_EVERY}.\n")
        f.write("# written by tests/golden/make_steady_state.py\n")
        f.write(f"# peak densities over {PEAK_NODES}x{PEAK_NODES}-node neighbourhoods, then "
                "over single nodes\n")
        f.write("# seed I_cath_A V_cath_V N_e N_i peak_ne_m3 peak_ni_m3 node_peak_ne_m3 "
                "node_peak_ni_m3\n")
        for r in rows:
            f.write(f"{r[0]:d} " + " ".join(f"{v:.10e}" for v in r[1:]) + "\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
