"""ctypes wrapper of the CPU oracle (test infrastructure only).

Marshals numpy arrays and parameter dictionaries into ``liboracle.so``; all
arithmetic is in oracle.c.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None


class OracleConfig(C.Structure):
    _fields_ = [
        ("nr", C.c_int32), ("nz", C.c_int32),
        ("R", C.c_double), ("L", C.c_double), ("Rc", C.c_double),
        ("dt", C.c_double), ("weight", C.c_double), ("m_ion", C.c_double),
        ("n_gas", C.c_double), ("T_gas", C.c_double),
        ("b_mode", C.c_int32),
        ("B_kA0", C.c_double), ("B_k", C.c_double), ("B0r", C.c_double), ("B0z", C.c_double),
        ("gamma_i", C.c_double), ("gamma_e", C.c_double),
        ("circuit_mode", C.c_int32),
        ("Vc_fixed", C.c_double), ("Vs", C.c_double), ("Rext", C.c_double),
        ("n_avg", C.c_int32), ("gather", C.c_int32), ("rweight", C.c_int32),
        ("mcc_on", C.c_int32), ("push_on", C.c_int32), ("field_on", C.c_int32),
        ("walls_reflect", C.c_int32),
        ("seed", C.c_uint64),
        ("sigma_el", C.c_double), ("ion_a", C.c_double), ("ion_I", C.c_double),
        ("exc_C", C.c_double), ("exc_E", C.c_double), ("E_cap", C.c_double),
        ("n_meta", C.c_double), ("meta_a", C.c_double), ("meta_I", C.c_double),
        ("gap_neumann", C.c_int32), ("wall_neumann", C.c_int32),
        ("band_r_lo", C.c_double), ("band_r_hi", C.c_double),
        ("ied_bins", C.c_int32), ("ied_emax", C.c_double),
    ]

    @classmethod
    def from_params(cls, p: dict) -> "OracleConfig":
        c = cls()
        for name, _ in cls._fields_:
            setattr(c, name, p[name])
        return c


class OracleDiag(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("t", "I_cath", "V_cath", "n_e_peak", "n_i_peak", "W_field", "K_e", "K_i")] + \
               [(n, C.c_int64) for n in
                ("N_e", "N_i", "n_ion_cath", "n_e_cath", "n_sey", "n_ionize", "n_excite",
                 "n_elastic", "n_ionize_meta", "ppc_max_e", "ppc_max_i")]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class OracleRegions(C.Structure):
    _fields_ = [("samples", C.c_int64), ("Te", C.c_double * 3), ("ncell", C.c_int64 * 3),
                ("z_sheath", C.c_double), ("z_bulk", C.c_double), ("ion_impacts", C.c_int64)]

    def as_dict(self) -> dict:
        return {"samples": self.samples, "Te": list(self.Te), "ncell": list(self.ncell),
                "z_sheath": self.z_sheath, "z_bulk": self.z_bulk,
                "ion_impacts": self.ion_impacts}


_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_U64 = C.POINTER(C.c_uint64)
_U32 = C.POINTER(C.c_uint32)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        cfgp = C.POINTER(OracleConfig)
        L.orc_philox4x64.argtypes = [_U64, _U64, _U64]
        L.orc_philox4x32.argtypes = [_U32, _U32, _U32]
        L.orc_boris_move.argtypes = [C.c_double] * 6 + [_D] * 5
        L.orc_bfield.argtypes = [cfgp, C.c_double, C.c_double, _D, _D]
        L.orc_node_volume.argtypes = [cfgp, C.c_int, C.c_int]
        L.orc_node_volume.restype = C.c_double
        L.orc_deposit.argtypes = [cfgp, C.c_int64, _D, _D, C.c_double, _D]
        L.orc_poisson.argtypes = [cfgp, _D, _D, _D]
        L.orc_efield_at.argtypes = [cfgp, _D, C.c_double, C.c_double, _D, _D]
        L.orc_sigma.argtypes = [cfgp, C.c_double, _D]
        L.orc_sigma_meta.argtypes = [cfgp, C.c_double]
        L.orc_sigma_meta.restype = C.c_double
        L.orc_nu_max.argtypes = [cfgp]
        L.orc_nu_max.restype = C.c_double
        L.orc_field_energy.argtypes = [cfgp, _D]
        L.orc_field_energy.restype = C.c_double
        L.orc_create.argtypes = [cfgp]
        L.orc_create.restype = C.c_void_p
        L.orc_set_particles.argtypes = [C.c_void_p, C.c_int, C.c_int64] + [_D] * 5 + [_I64]
        L.orc_count.argtypes = [C.c_void_p, C.c_int]
        L.orc_count.restype = C.c_int64
        L.orc_get_particles.argtypes = [C.c_void_p, C.c_int] + [_D] * 5 + [_I64]
        L.orc_solve_fields.argtypes = [C.c_void_p]
        L.orc_set_phi.argtypes = [C.c_void_p, _D]
        L.orc_get_fields.argtypes = [C.c_void_p, _D, _D, _D]
        L.orc_get_species_charge.argtypes = [C.c_void_p, C.c_int, _D]
        L.orc_set_circuit.argtypes = [C.c_void_p, C.c_double, C.c_int64, _D, C.c_int]
        L.orc_step.argtypes = [C.c_void_p, C.c_int64]
        L.orc_get_diag.argtypes = [C.c_void_p, C.POINTER(OracleDiag)]
        L.orc_set_next_id.argtypes = [C.c_void_p, C.c_int64]
        L.orc_get_next_id.argtypes = [C.c_void_p]
        L.orc_get_next_id.restype = C.c_int64
        L.orc_get_step.argtypes = [C.c_void_p]
        L.orc_get_step.restype = C.c_int64
        L.orc_reweight.argtypes = [C.c_void_p, C.c_int]
        L.orc_reweight.restype = C.c_int64
        L.orc_get_weight.argtypes = [C.c_void_p]
        L.orc_get_weight.restype = C.c_double
        L.orc_region_sample.argtypes = [C.c_void_p]
        L.orc_region_result.argtypes = [C.c_void_p, C.POINTER(OracleRegions), _D, _D]
        L.orc_ied_get.argtypes = [C.c_void_p, _I64, _I64]
        L.orc_region_reset.argtypes = [C.c_void_p]
        L.orc_destroy.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def philox4x64(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64(c.ctypes.data_as(_U64), k.ctypes.data_as(_U64), out.ctypes.data_as(_U64))
    return out


def philox4x32(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32), out.ctypes.data_as(_U32))
    return out


def boris_move(q_over_m, dt, Er, Ez, Br, Bz, state):
    """One push + move of a single particle; state = [r, z, vr, vt, vz]."""
    v = [C.c_double(x) for x in state]
    lib().orc_boris_move(q_over_m, dt, Er, Ez, Br, Bz, *[C.byref(x) for x in v])
    return np.array([x.value for x in v])


def bfield(p: dict, r: float, z: float):
    cfg = OracleConfig.from_params(p)
    br, bz = C.c_double(), C.c_double()
    lib().orc_bfield(C.byref(cfg), r, z, C.byref(br), C.byref(bz))
    return br.value, bz.value


def node_volume(p: dict) -> np.ndarray:
    cfg = OracleConfig.from_params(p)
    out = np.empty((p["nr"] + 1, p["nz"] + 1))
    for m in range(p["nr"] + 1):
        for n in range(p["nz"] + 1):
            out[m, n] = lib().orc_node_volume(C.byref(cfg), m, n)
    return out


def deposit(p: dict, r, z, qw: float) -> np.ndarray:
    cfg = OracleConfig.from_params(p)
    r, z = _f64(r), _f64(z)
    Q = np.zeros((p["nr"] + 1, p["nz"] + 1))
    lib().orc_deposit(C.byref(cfg), r.shape[0], _dp(r), _dp(z), qw, _dp(Q))
    return Q


def poisson(p: dict, rho, phi_bc) -> np.ndarray:
    cfg = OracleConfig.from_params(p)
    rho, phi_bc = _f64(rho), _f64(phi_bc)
    phi = np.zeros_like(rho)
    rc = lib().orc_poisson(C.byref(cfg), _dp(rho), _dp(phi_bc), _dp(phi))
    if rc != 0:
        raise RuntimeError(f"oracle poisson failed: {rc}")
    return phi


def efield_at(p: dict, phi, r: float, z: float):
    cfg = OracleConfig.from_params(p)
    phi = _f64(phi)
    er, ez = C.c_double(), C.c_double()
    lib().orc_efield_at(C.byref(cfg), _dp(phi), r, z, C.byref(er), C.byref(ez))
    return er.value, ez.value


def sigma(p: dict, E: float) -> np.ndarray:
    cfg = OracleConfig.from_params(p)
    out = np.zeros(3)
    lib().orc_sigma(C.byref(cfg), E, _dp(out))
    return out


def sigma_meta(p: dict, E: float) -> float:
    cfg = OracleConfig.from_params(p)
    return lib().orc_sigma_meta(C.byref(cfg), E)


def nu_max(p: dict) -> float:
    cfg = OracleConfig.from_params(p)
    return lib().orc_nu_max(C.byref(cfg))


def field_energy(p: dict, phi) -> float:
    cfg = OracleConfig.from_params(p)
    phi = _f64(phi)
    return lib().orc_field_energy(C.byref(cfg), _dp(phi))


class Oracle:
    """The time stepper.  ``particles`` = {"e": {...}, "i": {...}} of numpy arrays."""

    def __init__(self, params: dict, particles: dict | None = None, solve: bool = True):
        self.p = dict(params)
        self._cfg = OracleConfig.from_params(self.p)
        self._h = lib().orc_create(C.byref(self._cfg))
        if not self._h:
            raise RuntimeError("orc_create failed")
        if particles is not None:
            for k, sp in (("e", 0), ("i", 1)):
                self.set_particles(sp, particles[k])
            if solve:
                lib().orc_solve_fields(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    @property
    def shape(self):
        return (self.p["nr"] + 1, self.p["nz"] + 1)

    def set_particles(self, species: int, d: dict):
        arrs = [_f64(d[k]) for k in ("r", "z", "vr", "vt", "vz")]
        ids = np.ascontiguousarray(d["id"], dtype=np.int64)
        lib().orc_set_particles(self._h, species, ids.shape[0], *[_dp(a) for a in arrs],
                                ids.ctypes.data_as(_I64))

    def count(self, species: int) -> int:
        return lib().orc_count(self._h, species)

    def get_particles(self, species: int) -> dict:
        n = lib().orc_count(self._h, species)
        out = {k: np.empty(n) for k in ("r", "z", "vr", "vt", "vz")}
        out["id"] = np.empty(n, dtype=np.int64)
        lib().orc_get_particles(self._h, species, *[_dp(out[k]) for k in ("r", "z", "vr", "vt", "vz")],
                                out["id"].ctypes.data_as(_I64))
        return out

    def solve_fields(self):
        lib().orc_solve_fields(self._h)

    def set_phi(self, phi):
        phi = _f64(phi)
        lib().orc_set_phi(self._h, _dp(phi))

    def fields(self) -> dict:
        phi, rho, Q = (np.empty(self.shape) for _ in range(3))
        lib().orc_get_fields(self._h, _dp(phi), _dp(rho), _dp(Q))
        return {"phi": phi, "rho": rho, "Q": Q}

    def species_charge(self, species: int) -> np.ndarray:
        """Node charge (C) that one species deposited in the last step."""
        Q = np.empty(self.shape)
        lib().orc_get_species_charge(self._h, species, _dp(Q))
        return Q

    def set_circuit(self, Vc: float, step: int, qhist=None):
        q = _f64(qhist if qhist is not None else np.zeros(max(1, self.p["n_avg"])))
        lib().orc_set_circuit(self._h, Vc, step, _dp(q), q.shape[0])

    def step(self, n: int = 1):
        rc = lib().orc_step(self._h, n)
        if rc != 0:
            raise RuntimeError(f"oracle step failed: {rc}")

    def diag(self) -> dict:
        d = OracleDiag()
        lib().orc_get_diag(self._h, C.byref(d))
        return d.as_dict()

    @property
    def next_id(self) -> int:
        return lib().orc_get_next_id(self._h)

    @next_id.setter
    def next_id(self, v: int):
        lib().orc_set_next_id(self._h, v)

    @property
    def step_index(self) -> int:
        return lib().orc_get_step(self._h)

    def reweight(self, factor: int) -> int:
        """Keep each particle with probability 1/factor, weight x factor
        (Section 6); returns the particles kept."""
        kept = lib().orc_reweight(self._h, factor)
        if kept < 0:
            raise ValueError("factor must be >= 1")
        return kept

    @property
    def weight(self) -> float:
        return lib().orc_get_weight(self._h)

    def region_sample(self):
        lib().orc_region_sample(self._h)

    def regions(self) -> dict:
        """Region diagnostics of the accumulated samples (Sections 4, 5):
        dict with samples, Te[3], ncell[3], z_sheath, z_bulk, ion_impacts and
        the per-column edges zs, zb (nr values each)."""
        out = OracleRegions()
        zs, zb = np.zeros(self.p["nr"]), np.zeros(self.p["nr"])
        lib().orc_region_result(self._h, C.byref(out), _dp(zs), _dp(zb))
        d = out.as_dict()
        d["zs"], d["zb"] = zs, zb
        return d

    def ied(self):
        """Cathode ion energy histogram (Section 7) and its overflow count."""
        h = np.zeros(max(1, self.p["ied_bins"]), dtype=np.int64)
        over = C.c_int64()
        lib().orc_ied_get(self._h, h.ctypes.data_as(_I64), C.byref(over))
        return h[: self.p["ied_bins"]], over.value

    def region_reset(self):
        lib().orc_region_reset(self._h)
