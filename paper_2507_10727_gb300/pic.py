"""Thin ctypes binding of ``libpic_gb300.so`` (C ABI in ``include/pic.h``).

Functions carry the C names and only marshal arguments: parameter dicts into
``pic_config``, numpy arrays or torch tensors into pointers, torch's caching
allocator and current CUDA stream into ``pic_alloc`` / ``cudaStream_t``.  All
computation runs in the library's CUDA kernels; there is no fallback: if the
library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic_gb300.so")

PIC_OK = 0
ERRORS = {
    -1: "PIC_ERR_INVALID", -2: "PIC_ERR_OOM", -3: "PIC_ERR_CAPACITY",
    -4: "PIC_ERR_NONCONVERGED", -5: "PIC_ERR_NAN", -6: "PIC_ERR_TIMEOUT",
    -7: "PIC_ERR_CUDA", -8: "PIC_ERR_IO",
}


class PicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class PicConfig(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("nr", C.c_int32), ("nz", C.c_int32),
        ("R", C.c_double), ("L", C.c_double), ("Rc", C.c_double), ("dt", C.c_double),
        ("weight", C.c_double), ("m_ion", C.c_double), ("n_gas", C.c_double),
        ("T_gas", C.c_double),
        ("b_mode", C.c_int32),
        ("B_kA0", C.c_double), ("B_k", C.c_double), ("B0r", C.c_double), ("B0z", C.c_double),
        ("gamma_i", C.c_double), ("gamma_e", C.c_double),
        ("circuit_mode", C.c_int32),
        ("Vc_fixed", C.c_double), ("Vs", C.c_double), ("Rext", C.c_double),
        ("n_avg", C.c_int32), ("gather", C.c_int32), ("rweight", C.c_int32),
        ("precision", C.c_int32), ("mcc_on", C.c_int32), ("push_on", C.c_int32),
        ("field_on", C.c_int32), ("walls_reflect", C.c_int32),
        ("seed", C.c_uint64),
        ("sigma_el", C.c_double), ("ion_a", C.c_double), ("ion_I", C.c_double),
        ("exc_C", C.c_double), ("exc_E", C.c_double), ("E_cap", C.c_double),
        ("poisson_tol", C.c_double), ("poisson_max_iter", C.c_int32),
        ("cap_e", C.c_int64), ("cap_i", C.c_int64), ("birth_cap", C.c_int64),
        ("diag_every", C.c_int32), ("sort_every", C.c_int32),
        ("n_meta", C.c_double), ("meta_a", C.c_double), ("meta_I", C.c_double),
        ("gap_neumann", C.c_int32), ("wall_neumann", C.c_int32),
        ("band_r_lo", C.c_double), ("band_r_hi", C.c_double),
        ("ied_bins", C.c_int32), ("ied_emax", C.c_double), ("phi_extrapolate", C.c_int32),
        ("poisson_precond", C.c_int32),
    ]

    @classmethod
    def from_params(cls, p: dict) -> "PicConfig":
        c = cls()
        for name, _ in cls._fields_:
            if name == "struct_size":
                continue
            setattr(c, name, p[name])
        c.struct_size = C.sizeof(cls)
        return c


class PicDiag(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("t", "I_cath", "V_cath", "n_e_peak", "n_i_peak", "W_field", "K_e", "K_i")] + \
               [(n, C.c_int64) for n in
                ("N_e", "N_i", "n_ion_cath", "n_e_cath", "n_sey", "n_ionize", "n_excite",
                 "n_elastic", "step", "particle_steps")] + \
               [("poisson_iters", C.c_int32), ("status", C.c_int32),
                ("poisson_resid", C.c_double), ("n_ionize_meta", C.c_int64),
                ("ppc_max_e", C.c_int64), ("ppc_max_i", C.c_int64), ("weight", C.c_double)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class PicRegions(C.Structure):
    _fields_ = [("samples", C.c_int64), ("Te", C.c_double * 3), ("ncell", C.c_int64 * 3),
                ("z_sheath", C.c_double), ("z_bulk", C.c_double), ("ion_impacts", C.c_int64)]

    def as_dict(self) -> dict:
        return {"samples": self.samples, "Te": list(self.Te), "ncell": list(self.ncell),
                "z_sheath": self.z_sheath, "z_bulk": self.z_bulk,
                "ion_impacts": self.ion_impacts}


class PicUnetStats(C.Structure):
    _fields_ = [("snapshots", C.c_int64), ("starts_previous", C.c_int64),
                ("starts_network", C.c_int64), ("starts_zero", C.c_int64),
                ("poisson_iters", C.c_int64), ("in_norm", C.c_double), ("out_norm", C.c_double),
                ("last_start", C.c_int32), ("pad", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class PicKernelTime(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_int64), ("total_ms", C.c_double)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class PicAlloc(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", _ALLOC_FN), ("free", _FREE_FN)]


_lib = None
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build()")
        L = C.CDLL(path)
        vp = C.c_void_p
        L.pic_create.argtypes = [C.POINTER(PicConfig), C.c_int, C.POINTER(PicAlloc), vp,
                                 C.POINTER(vp)]
        L.pic_destroy.argtypes = [vp]
        L.pic_destroy.restype = None
        L.pic_last_error.argtypes = [vp]
        L.pic_last_error.restype = C.c_char_p
        L.pic_set_particles.argtypes = [vp, C.c_int, C.c_int, C.c_int64] + [vp] * 6 + [C.c_int]
        L.pic_count.argtypes = [vp, C.c_int, C.c_int, _I64]
        L.pic_get_particles.argtypes = [vp, C.c_int, C.c_int] + [vp] * 6 + [C.c_int]
        L.pic_solve_fields.argtypes = [vp, C.c_int]
        L.pic_set_phi.argtypes = [vp, C.c_int, vp, C.c_int]
        L.pic_get_fields.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int]
        L.pic_set_circuit.argtypes = [vp, C.c_int, C.c_double, C.c_int64, _D, C.c_int]
        L.pic_set_next_id.argtypes = [vp, C.c_int, C.c_int64]
        L.pic_get_next_id.argtypes = [vp, C.c_int, _I64]
        L.pic_step.argtypes = [vp, C.c_int64]
        L.pic_uses_graph.argtypes = [vp]
        L.pic_tuned_chunk.argtypes = [vp, C.POINTER(C.c_int)]
        L.pic_set_chunk.argtypes = [vp, C.c_int]
        L.pic_set_tile.argtypes = [vp, C.c_int]
        L.pic_fp64_fma_rate.argtypes = [vp, _D]
        L.pic_tuned_tile.argtypes = [vp, C.POINTER(C.c_int)]
        L.pic_autotune_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), _I64]
        L.pic_get_species_charge.argtypes = [vp, C.c_int, C.c_int, vp, C.c_int]
        L.pic_sync.argtypes = [vp]
        L.pic_diagnostics.argtypes = [vp, C.c_int, C.POINTER(PicDiag)]
        L.pic_reweight.argtypes = [vp, C.c_int, C.c_int]
        L.pic_region_sample.argtypes = [vp, C.c_int]
        L.pic_region_read.argtypes = [vp, C.c_int, C.POINTER(PicRegions), vp, vp, vp, _I64]
        L.pic_region_reset.argtypes = [vp, C.c_int]
        L.pic_save.argtypes = [vp, C.c_int, C.c_char_p]
        L.pic_load.argtypes = [vp, C.c_int, C.c_char_p]
        L.pic_profile.argtypes = [vp, C.c_int]
        L.pic_profile_read.argtypes = [vp, C.POINTER(PicKernelTime), C.c_int,
                                       C.POINTER(C.c_int)]
        L.pic_unet_param_count.argtypes = [_I64]
        L.pic_unet_create.argtypes = [vp, C.c_uint64, C.c_int, C.c_int]
        L.pic_unet_set_params.argtypes = [vp, vp, C.c_int64]
        L.pic_unet_get_params.argtypes = [vp, vp, C.c_int64]
        L.pic_unet_loss_grad.argtypes = [vp, C.c_int, vp, vp, vp, vp, _D]
        L.pic_unet_snapshots.argtypes = [vp, C.c_int64, C.c_int]
        L.pic_unet_train.argtypes = [vp, C.c_int, C.c_int, C.c_float, C.c_uint64, _D, _D]
        L.pic_unet_warm_start.argtypes = [vp, C.c_int]
        L.pic_unet_set_norms.argtypes = [vp, C.c_double, C.c_double]
        L.pic_unet_record.argtypes = [vp, C.c_int]
        L.pic_unet_stats_read.argtypes = [vp, C.POINTER(PicUnetStats)]
        L.pic_poisson_workspace_bytes.argtypes = [C.c_int, C.c_int]
        L.pic_poisson_workspace_bytes.restype = C.c_size_t
        L.pic_poisson_solve.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                        C.c_int, vp, vp, vp, vp, C.POINTER(C.c_int), _D]
        L.pic_poisson_solve_mixed.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                              C.c_int, C.c_double, C.c_int, vp, vp, vp, vp,
                                              C.POINTER(C.c_int), _D]
        _lib = L
    return _lib


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the PIC library runs on the GPU only")
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


_live = weakref.WeakSet()


class Handle:
    """Owns a ``pic_handle*`` plus the allocator callbacks that must stay alive."""

    def __init__(self, ptr: int, keep: tuple, n_instances: int, params: list[dict]):
        self.ptr = ptr
        self._keep = keep
        self.n_instances = n_instances
        self.params = params
        _live.add(self)

    def __del__(self):
        if getattr(self, "ptr", None):
            load_library().pic_destroy(self.ptr)
            self.ptr = None


@atexit.register
def _destroy_live_handles():
    # release device memory while torch's allocator is still alive
    for h in list(_live):
        if h.ptr:
            load_library().pic_destroy(h.ptr)
            h.ptr = None


def _check(h, rc: int):
    if rc != PIC_OK:
        msg = load_library().pic_last_error(h.ptr if isinstance(h, Handle) else h) or b""
        raise PicError(rc, msg.decode())


def pic_create(params, stream=None, torch_alloc: bool = True) -> Handle:
    """Create a handle for one parameter dict or a list of them (instances)."""
    torch = _torch()
    L = load_library()
    plist = params if isinstance(params, (list, tuple)) else [params]
    cfgs = (PicConfig * len(plist))(*[PicConfig.from_params(p) for p in plist])
    keep = ()
    alloc_p = None
    if torch_alloc:
        dev = torch.cuda.current_device()
        s = stream if stream is not None else torch.cuda.current_stream()

        def _alloc(ctx, nbytes):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, s)
            except RuntimeError:
                return None

        def _free(ctx, ptr):
            torch.cuda.caching_allocator_delete(ptr)

        fa, ff = _ALLOC_FN(_alloc), _FREE_FN(_free)
        alloc = PicAlloc(None, fa, ff)
        keep = (fa, ff, alloc)
        alloc_p = C.byref(alloc)
    out = C.c_void_p()
    rc = L.pic_create(cfgs, len(plist), alloc_p, _stream_ptr(stream), C.byref(out))
    if rc != PIC_OK:
        raise PicError(rc, "pic_create failed (invalid configuration or allocation)")
    return Handle(out.value, keep, len(plist), [dict(p) for p in plist])


def pic_destroy(h: Handle):
    if h.ptr:
        load_library().pic_destroy(h.ptr)
        h.ptr = None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def pic_set_particles(h: Handle, instance: int, species: int, d: dict):
    """Load particles from host arrays (numpy arrays or CPU tensors, passed
    without a copy: page-locked memory, e.g. a tensor's pin_memory(), is read
    in place by the load kernels) or CUDA tensors (device)."""
    keys = ("r", "z", "vr", "vt", "vz")
    first = d["r"]
    if hasattr(first, "is_cuda") and first.is_cuda:
        ts = [d[k].contiguous() for k in keys] + [d["id"].contiguous()]
        n = ts[0].numel()
        ptrs = [t.data_ptr() for t in ts]
        rc = load_library().pic_set_particles(h.ptr, instance, species, n, *ptrs, 1)
    else:
        arrs = [_f64(d[k]) for k in keys] + [np.ascontiguousarray(d["id"], dtype=np.int64)]
        n = arrs[0].shape[0]
        rc = load_library().pic_set_particles(h.ptr, instance, species, n,
                                              *[a.ctypes.data for a in arrs], 0)
    _check(h, rc)


def pic_count(h: Handle, instance: int, species: int) -> int:
    n = C.c_int64()
    _check(h, load_library().pic_count(h.ptr, instance, species, C.byref(n)))
    return n.value


def pic_get_particles(h: Handle, instance: int, species: int) -> dict:
    n = pic_count(h, instance, species)
    out = {k: np.empty(n) for k in ("r", "z", "vr", "vt", "vz")}
    out["id"] = np.empty(n, dtype=np.int64)
    rc = load_library().pic_get_particles(
        h.ptr, instance, species, *[out[k].ctypes.data for k in ("r", "z", "vr", "vt", "vz", "id")], 0)
    _check(h, rc)
    return out


def _node_shape(h: Handle, instance: int):
    p = h.params[instance]
    return (p["nr"] + 1, p["nz"] + 1)


def pic_solve_fields(h: Handle, instance: int = 0):
    _check(h, load_library().pic_solve_fields(h.ptr, instance))


def pic_set_phi(h: Handle, instance: int, phi):
    a = _f64(phi)
    assert a.shape == _node_shape(h, instance)
    _check(h, load_library().pic_set_phi(h.ptr, instance, a.ctypes.data, 0))


def pic_get_fields(h: Handle, instance: int = 0) -> dict:
    shp = _node_shape(h, instance)
    phi, rho, Q = np.empty(shp), np.empty(shp), np.empty(shp)
    rc = load_library().pic_get_fields(h.ptr, instance, phi.ctypes.data, rho.ctypes.data,
                                       Q.ctypes.data, 0)
    _check(h, rc)
    return {"phi": phi, "rho": rho, "Q": Q}


def pic_get_species_charge(h: Handle, instance: int, species: int) -> np.ndarray:
    Q = np.empty(_node_shape(h, instance))
    _check(h, load_library().pic_get_species_charge(h.ptr, instance, species, Q.ctypes.data, 0))
    return Q


def pic_set_circuit(h: Handle, instance: int, Vc: float, step: int, qhist=None):
    q = _f64(qhist if qhist is not None else np.zeros(h.params[instance]["n_avg"]))
    _check(h, load_library().pic_set_circuit(h.ptr, instance, Vc, step,
                                             q.ctypes.data_as(_D), q.shape[0]))


def pic_set_next_id(h: Handle, instance: int, next_id: int):
    _check(h, load_library().pic_set_next_id(h.ptr, instance, next_id))


def pic_get_next_id(h: Handle, instance: int = 0) -> int:
    v = C.c_int64()
    _check(h, load_library().pic_get_next_id(h.ptr, instance, C.byref(v)))
    return v.value


def pic_step(h: Handle, nsteps: int = 1):
    _check(h, load_library().pic_step(h.ptr, nsteps))


def pic_uses_graph(h: Handle) -> bool:
    return bool(load_library().pic_uses_graph(h.ptr))


def pic_tuned_chunk(h: Handle) -> int:
    v = C.c_int()
    _check(h, load_library().pic_tuned_chunk(h.ptr, C.byref(v)))
    return v.value


def pic_fp64_fma_rate(stream=None) -> float:
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    v = C.c_double(0.0)
    rc = load_library().pic_fp64_fma_rate(C.c_void_p(st.cuda_stream), C.byref(v))
    if rc != 0:
        raise PicError(rc, "pic_fp64_fma_rate")
    return v.value


def pic_set_tile(h: Handle, shape: int = 0):
    """Cell tile shape: 1 = 8 x 8, 2 = 16 x 8, 3 = 8 x 16 (r x z) fixed; 0 = autotuned."""
    _check(h, load_library().pic_set_tile(h.ptr, int(shape)))


def pic_tuned_tile(h: Handle) -> int:
    v = C.c_int(0)
    _check(h, load_library().pic_tuned_tile(h.ptr, C.byref(v)))
    return v.value


def pic_set_chunk(h: Handle, particles_per_thread: int):
    _check(h, load_library().pic_set_chunk(h.ptr, particles_per_thread))


def pic_autotune_info(h: Handle) -> dict:
    t, ppt, n = C.c_int(), C.c_int(), C.c_int64()
    _check(h, load_library().pic_autotune_info(h.ptr, C.byref(t), C.byref(ppt), C.byref(n)))
    return {"tunings": t.value, "particles_per_thread": ppt.value, "particles_at_tuning": n.value}


def pic_sync(h: Handle):
    _check(h, load_library().pic_sync(h.ptr))


def pic_diagnostics(h: Handle, instance: int = 0, check: bool = True) -> dict:
    d = PicDiag()
    rc = load_library().pic_diagnostics(h.ptr, instance, C.byref(d))
    if check:
        _check(h, rc)
    return d.as_dict()


def pic_reweight(h: Handle, instance: int, factor: int = 3):
    _check(h, load_library().pic_reweight(h.ptr, instance, factor))


def pic_region_sample(h: Handle, instance: int = 0):
    _check(h, load_library().pic_region_sample(h.ptr, instance))


def pic_region_read(h: Handle, instance: int = 0) -> dict:
    """Region diagnostics of the accumulated samples and the cathode ion
    energy histogram: dict as PicRegions plus zs, zb (per cell column) and
    ied, ied_overflow."""
    nr = h.params[instance]["nr"]
    bins = h.params[instance].get("ied_bins", 0)
    out = PicRegions()
    zs, zb = np.zeros(nr), np.zeros(nr)
    ied = np.zeros(max(1, bins), dtype=np.int64)
    over = C.c_int64()
    _check(h, load_library().pic_region_read(h.ptr, instance, C.byref(out),
                                             zs.ctypes.data, zb.ctypes.data, ied.ctypes.data,
                                             C.byref(over)))
    d = out.as_dict()
    d.update(zs=zs, zb=zb, ied=ied[:bins], ied_overflow=over.value)
    return d


def pic_region_reset(h: Handle, instance: int = 0):
    _check(h, load_library().pic_region_reset(h.ptr, instance))


def pic_save(h: Handle, instance: int, path: str):
    _check(h, load_library().pic_save(h.ptr, instance, path.encode()))


def pic_load(h: Handle, instance: int, path: str):
    _check(h, load_library().pic_load(h.ptr, instance, path.encode()))


def pic_profile(h: Handle, enable: bool):
    _check(h, load_library().pic_profile(h.ptr, 1 if enable else 0))


def pic_profile_read(h: Handle) -> dict:
    arr = (PicKernelTime * 32)()
    n = C.c_int()
    _check(h, load_library().pic_profile_read(h.ptr, arr, 32, C.byref(n)))
    return {arr[k].name.decode(): {"launches": arr[k].launches, "total_ms": arr[k].total_ms}
            for k in range(n.value)}


def pic_poisson_workspace_bytes(nr: int, nz: int) -> int:
    return load_library().pic_poisson_workspace_bytes(nr, nz)


def pic_poisson_solve(nr: int, nz: int, R: float, L: float, tol: float, max_iter: int, Q, phi,
                      work=None, stream=None, first_insulating_z0=None, wall_insulating=0):
    """Solve in place on CUDA tensors Q, phi ((nr+1) x (nz+1) float64).  With
    ``first_insulating_z0`` or ``wall_insulating`` set, pic_poisson_solve_mixed
    (insulating boundary parts) is called."""
    torch = _torch()
    if work is None:
        work = torch.empty(pic_poisson_workspace_bytes(nr, nz), dtype=torch.uint8, device=Q.device)
    it = C.c_int()
    res = C.c_double()
    if first_insulating_z0 is None and not wall_insulating:
        rc = load_library().pic_poisson_solve(nr, nz, R, L, tol, max_iter, Q.data_ptr(),
                                              phi.data_ptr(), work.data_ptr(), _stream_ptr(stream),
                                              C.byref(it), C.byref(res))
    else:
        g = nr + 1 if first_insulating_z0 is None else first_insulating_z0
        rc = load_library().pic_poisson_solve_mixed(nr, nz, R, L, g, int(wall_insulating), tol,
                                                    max_iter, Q.data_ptr(), phi.data_ptr(),
                                                    work.data_ptr(), _stream_ptr(stream),
                                                    C.byref(it), C.byref(res))
    if rc != PIC_OK and rc != -4:
        raise PicError(rc, "pic_poisson_solve failed")
    return rc, it.value, res.value


# ---------------------------------------------------------------------------
# learned warm start
# ---------------------------------------------------------------------------
def pic_unet_param_count() -> int:
    n = C.c_int64()
    rc = load_library().pic_unet_param_count(C.byref(n))
    if rc != PIC_OK:
        raise PicError(rc, "pic_unet_param_count")
    return n.value


def pic_unet_create(h: Handle, seed: int = 0, max_batch: int = 1, mode: int = 0):
    _check(h, load_library().pic_unet_create(h.ptr, seed, max_batch, mode))


def pic_unet_set_params(h: Handle, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(h, load_library().pic_unet_set_params(h.ptr, p.ctypes.data, p.size))


def pic_unet_get_params(h: Handle) -> np.ndarray:
    p = np.empty(pic_unet_param_count(), dtype=np.float32)
    _check(h, load_library().pic_unet_get_params(h.ptr, p.ctypes.data, p.size))
    return p


def pic_unet_loss_grad(h: Handle, x, y=None):
    """x: (B, 3, nr+1, nz+1), y: (B, nr+1, nz+1) or None.  Returns
    (out (B, nr+1, nz+1), grad or None, loss or None) as FP32 numpy / float."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    B, _, H, W = x.shape
    out = np.empty((B, H, W), dtype=np.float32)
    yp = gp = 0
    grad = None
    loss = C.c_double()
    if y is not None:
        y = np.ascontiguousarray(y, dtype=np.float32).reshape(B, H, W)
        grad = np.empty(pic_unet_param_count(), dtype=np.float32)
        yp, gp = y.ctypes.data, grad.ctypes.data
    _check(h, load_library().pic_unet_loss_grad(h.ptr, B, x.ctypes.data, yp or None,
                                                out.ctypes.data, gp or None, C.byref(loss)))
    return out, grad, (loss.value if y is not None else None)


def pic_unet_snapshots(h: Handle, capacity: int, every: int = 1):
    _check(h, load_library().pic_unet_snapshots(h.ptr, capacity, every))


def pic_unet_train(h: Handle, iters: int, batch: int, lr: float, seed: int = 0):
    a, b = C.c_double(), C.c_double()
    _check(h, load_library().pic_unet_train(h.ptr, iters, batch, lr, seed, C.byref(a), C.byref(b)))
    return a.value, b.value


def pic_unet_record(h: Handle, on: bool = True):
    _check(h, load_library().pic_unet_record(h.ptr, 1 if on else 0))


def pic_unet_set_norms(h: Handle, in_norm: float, out_norm: float):
    _check(h, load_library().pic_unet_set_norms(h.ptr, float(in_norm), float(out_norm)))


def pic_unet_warm_start(h: Handle, on: bool = True):
    _check(h, load_library().pic_unet_warm_start(h.ptr, 1 if on else 0))


def pic_unet_stats(h: Handle) -> dict:
    s = PicUnetStats()
    _check(h, load_library().pic_unet_stats_read(h.ptr, C.byref(s)))
    return s.as_dict()
