"""Python binding of the C ABI in include/rt.h (argument marshalling only).

Every function has the C name and forwards to `librt_b300.so`; all work runs
in the library's CUDA kernels. Host buffers are numpy arrays (or CPU torch
tensors); device buffers are CUDA torch tensors. There is no CPU fallback: if
the library is missing the import of the first call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

RT_OK, RT_E_INVAL, RT_E_STATE, RT_E_CUDA, RT_E_OOM, RT_E_BUDGET, RT_E_BOUNDS = 0, -1, -2, -3, -4, -5, -6
RT_HOST, RT_DEVICE = 0, 1
RT_PCLD_SCATTERING, RT_PCLD_EXTINCTION = 0, 1
RT_TALLY_FP64, RT_TALLY_FP32 = 0, 1
RT_OPTICS_SPLIT, RT_OPTICS_TOTAL = 0, 1
RT_HOM_SURFACE, RT_HOM_HEATING = 1, 2
RT_BIRTH_PHILOX, RT_BIRTH_SOBOL = 0, 1
RT_SCHEDULE_IDS, RT_SCHEDULE_THICK_FIRST = 0, 1

_ERRNAMES = {RT_E_INVAL: "RT_E_INVAL", RT_E_STATE: "RT_E_STATE", RT_E_CUDA: "RT_E_CUDA",
             RT_E_OOM: "RT_E_OOM", RT_E_BUDGET: "RT_E_BUDGET",
             RT_E_BOUNDS: "RT_E_BOUNDS"}


class RtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class rt_options(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("refill_chunk", ctypes.c_int), ("max_steps", ctypes.c_uint32),
                ("pcld_mode", ctypes.c_int), ("tally_precision", ctypes.c_int),
                ("ready_threshold", ctypes.c_int), ("max_inner", ctypes.c_int),
                ("batch_optics", ctypes.c_int), ("birth", ctypes.c_int), ("schedule", ctypes.c_int),
                ("box_levels", ctypes.c_int), ("box_tau", ctypes.c_float), ("tally_aggregate", ctypes.c_int),
                ("refill_min", ctypes.c_int)]


class rt_job(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_void_p), ("sza_deg", ctypes.c_double), ("azimuth_deg", ctypes.c_double),
                ("toa_flux", ctypes.c_double), ("gas_scale", ctypes.c_double), ("photons", ctypes.c_uint64),
                ("diffuse_fraction", ctypes.c_double)]


class rt_step_desc(ctypes.Structure):
    _fields_ = [("optics", ctypes.c_int), ("field", ctypes.c_void_p * 5), ("albedo", ctypes.c_void_p),
                ("photons", ctypes.c_uint64), ("abs3d", ctypes.c_void_p), ("hr", ctypes.c_void_p),
                ("sfc_dir", ctypes.c_void_p), ("sfc_dif", ctypes.c_void_p), ("toa_up", ctypes.c_void_p),
                ("homogenize", ctypes.c_int)]


class rt_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("photons", "events", "scatters", "crossings",
                                               "surface_hits", "roulette_kills", "capped",
                                               "max_events_photon")] + \
               [(n, ctypes.c_double) for n in ("energy_in", "energy_toa_up", "energy_atm_abs",
                                               "energy_sfc_abs", "energy_created",
                                               "energy_destroyed", "energy_capped")] + \
               [("status", ctypes.c_int)]


_lib = None


def library() -> ctypes.CDLL:
    """Load librt_b300.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is not built; run paper_2208_05247_b300.build.build(). "
                               "The tracer has no CPU fallback.")
        lib = ctypes.CDLL(LIB)
        H, P, i32, u64, f64 = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
        sig = {
            "rt_create": ([i32, i32, i32, f64, f64, f64], H),
            "rt_destroy": ([H], i32),
            "rt_set_stream": ([H, P], i32),
            "rt_set_options": ([H, ctypes.POINTER(rt_options)], i32),
            "rt_get_options": ([H, ctypes.POINTER(rt_options)], i32),
            "rt_set_optics": ([H, P, P, P, P, P, i32], i32),
            "rt_set_surface": ([H, P, i32], i32),
            "rt_build_accel": ([H, i32, i32, i32], i32),
            "rt_trace": ([H, f64, f64, f64, u64, u64], i32),
            "rt_trace_range": ([H, f64, f64, f64, u64, u64, u64, u64], i32),
            "rt_trace_ex": ([H, f64, f64, f64, f64, u64, u64, u64, u64], i32),
            "rt_set_optics_total": ([H, P, P, P, P, i32], i32),
            "rt_fields": ([H, P, P, P, P, i32], i32),
            "rt_fields_split": ([H, P, P, P, i32], i32),
            "rt_heating_rate": ([H, P, i32, i32], i32),
            "rt_trace_batch": ([ctypes.POINTER(rt_job), i32, u64, u64], i32),
            "rt_reset_tallies": ([H], i32),
            "rt_stats": ([H, ctypes.POINTER(rt_stats_t)], i32),
            "rt_synchronize": ([H], i32),
            "rt_last_error": ([], ctypes.c_char_p),
            "rt_last_error_code": ([], i32),
            "rt_trace_noalloc": ([i32, i32, i32, f64, f64, f64] + [P] * 6 + [i32, i32, i32, f64, f64, f64,
                                                                            u64, u64] + [P] * 5 + [P, P], i32),
            "rt_batch_step_create": ([ctypes.POINTER(rt_job), i32, u64, ctypes.POINTER(ctypes.c_void_p)], i32),
            "rt_batch_step_launch": ([P, u64], i32),
            "rt_batch_step_destroy": ([P], i32),
            "rt_step_create": ([H, ctypes.POINTER(rt_step_desc), ctypes.POINTER(ctypes.c_void_p)], i32),
            "rt_step_launch": ([P, f64, f64, f64, f64, u64], i32),
            "rt_step_destroy": ([P], i32),
            "rt_debug_philox": ([P, P, P, i32], i32),
            "rt_debug_sample": ([i32, ctypes.c_float, u64, u64, P], i32),
            "rt_debug_turn": ([P, P, P, P, i32], i32),
            "rt_debug_sobol": ([u64, i32, ctypes.c_uint32, ctypes.c_uint32, P], i32),
            "rt_probe_read": ([P, u64, i32, P, P], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def rt_last_error() -> str:
    return library().rt_last_error().decode()


def rt_last_error_code() -> int:
    return library().rt_last_error_code()


def _check(rc: int) -> int:
    if rc != RT_OK:
        raise RtError(rc, rt_last_error())
    return rc


def _buf(x, n: int | None, dtype, name: str, writable: bool = False):
    """(pointer, mem) of a numpy array or torch tensor with n elements of dtype."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags.c_contiguous or (writable and not x.flags.writeable):
            raise ValueError(f"{name}: need a C-contiguous {np.dtype(dtype).name} array")
        if n is not None and x.size != n:
            raise ValueError(f"{name}: expected {n} elements, got {x.size}")
        return x.ctypes.data, RT_HOST
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        want = {np.float32: torch.float32, np.float64: torch.float64}[np.dtype(dtype).type]
        if x.dtype != want or not x.is_contiguous():
            raise ValueError(f"{name}: need a contiguous {want} tensor")
        if n is not None and x.numel() != n:
            raise ValueError(f"{name}: expected {n} elements, got {x.numel()}")
        return x.data_ptr(), (RT_DEVICE if x.is_cuda else RT_HOST)
    raise TypeError(f"{name}: expected numpy array or torch tensor, got {type(x)}")


def _same_mem(*pairs):
    mems = {m for _, m in pairs if m is not None}
    if len(mems) > 1:
        raise ValueError("all buffers of one call must be host or all device")
    return mems.pop() if mems else RT_HOST


# ---- the C ABI, one function each -------------------------------------------------

def rt_create(nx, ny, nz, dx, dy, dz) -> int:
    h = library().rt_create(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz))
    if not h:
        raise RtError(rt_last_error_code(), rt_last_error())
    return h


def rt_destroy(h):
    return _check(library().rt_destroy(h))


def rt_set_stream(h, stream=None):
    if stream is None:
        ptr = None
    elif isinstance(stream, int):
        ptr = stream
    else:
        ptr = stream.cuda_stream
    return _check(library().rt_set_stream(h, ptr))


def rt_set_options(h, **kw):
    o = rt_options()
    _check(library().rt_get_options(h, ctypes.byref(o)))
    types = dict(rt_options._fields_)
    for k, v in kw.items():
        if k not in types:
            raise KeyError(k)
        setattr(o, k, float(v) if types[k] is ctypes.c_float else int(v))
    return _check(library().rt_set_options(h, ctypes.byref(o)))


def rt_get_options(h) -> dict:
    o = rt_options()
    _check(library().rt_get_options(h, ctypes.byref(o)))
    return {k: getattr(o, k) for k, _ in rt_options._fields_}


def rt_set_optics(h, ncell, k_gas, ssa_gas, k_cld, ssa_cld, g_cld):
    bufs = [_buf(a, ncell, np.float32, n) for a, n in
            zip((k_gas, ssa_gas, k_cld, ssa_cld, g_cld), ("k_gas", "ssa_gas", "k_cld", "ssa_cld", "g_cld"))]
    mem = _same_mem(*bufs)
    return _check(library().rt_set_optics(h, *[p for p, _ in bufs], mem))


def rt_set_optics_total(h, ncell, k_ext, k_ext_cld, ssa, g_cld):
    bufs = [_buf(a, ncell, np.float32, n) for a, n in
            zip((k_ext, k_ext_cld, ssa, g_cld), ("k_ext", "k_ext_cld", "ssa", "g_cld"))]
    mem = _same_mem(*bufs)
    return _check(library().rt_set_optics_total(h, *[p for p, _ in bufs], mem))


def rt_trace_ex(h, sza_deg, azimuth_deg, toa_flux, diffuse_fraction, photon_begin, photon_count, photons_total,
                seed):
    return _check(library().rt_trace_ex(h, float(sza_deg), float(azimuth_deg), float(toa_flux),
                                        float(diffuse_fraction), int(photon_begin), int(photon_count),
                                        int(photons_total), int(seed) & 0xFFFFFFFFFFFFFFFF))


def rt_set_surface(h, ncol, albedo):
    p, mem = _buf(albedo, ncol, np.float32, "albedo")
    return _check(library().rt_set_surface(h, p, mem))


def rt_build_accel(h, cx=0, cy=0, cz=0):
    return _check(library().rt_build_accel(h, int(cx), int(cy), int(cz)))


def rt_trace(h, sza_deg, azimuth_deg, toa_flux, photons, seed):
    return _check(library().rt_trace(h, float(sza_deg), float(azimuth_deg), float(toa_flux),
                                     int(photons), int(seed) & 0xFFFFFFFFFFFFFFFF))


def rt_trace_range(h, sza_deg, azimuth_deg, toa_flux, photon_begin, photon_count, photons_total, seed):
    return _check(library().rt_trace_range(h, float(sza_deg), float(azimuth_deg), float(toa_flux),
                                           int(photon_begin), int(photon_count), int(photons_total),
                                           int(seed) & 0xFFFFFFFFFFFFFFFF))


def rt_trace_batch(jobs, total_photons=0, seed=1):
    """jobs: sequence of dicts with scene (handle or Tracer), sza_deg, azimuth_deg,
    toa_flux, gas_scale and photons (used when total_photons is 0)."""
    arr = _job_array(jobs)
    return _check(library().rt_trace_batch(arr, len(jobs), int(total_photons), int(seed) & 0xFFFFFFFFFFFFFFFF))


def _job_array(jobs):
    arr = (rt_job * len(jobs))()
    for a, j in zip(arr, jobs):
        sc = j["scene"]
        a.scene = sc.h if hasattr(sc, "h") else sc
        a.sza_deg = float(j.get("sza_deg", 0.0))
        a.azimuth_deg = float(j.get("azimuth_deg", 0.0))
        a.toa_flux = float(j.get("toa_flux", 0.0))
        a.gas_scale = float(j.get("gas_scale", 1.0))
        a.photons = int(j.get("photons", 0))
        a.diffuse_fraction = float(j.get("diffuse_fraction", 0.0))
    return arr


def rt_batch_step_create(jobs, total_photons=0) -> int:
    """Record rt_trace_batch(jobs, total_photons) as one CUDA graph; returns the step."""
    out = ctypes.c_void_p(0)
    _check(library().rt_batch_step_create(_job_array(jobs), len(jobs), int(total_photons), ctypes.byref(out)))
    return out.value


def rt_batch_step_launch(step, seed=1):
    _check(library().rt_batch_step_launch(step, int(seed) & 0xFFFFFFFFFFFFFFFF))


def rt_batch_step_destroy(step):
    _check(library().rt_batch_step_destroy(step))


def rt_fields(h, ncell, ncol, abs3d=None, sfc_dir=None, sfc_dif=None, toa_up=None):
    bufs = [_buf(abs3d, ncell, np.float64, "abs3d", True), _buf(sfc_dir, ncol, np.float64, "sfc_dir", True),
            _buf(sfc_dif, ncol, np.float64, "sfc_dif", True), _buf(toa_up, ncol, np.float64, "toa_up", True)]
    mem = _same_mem(*bufs)
    return _check(library().rt_fields(h, *[p for p, _ in bufs], mem))


def rt_fields_split(h, ncell, ncol, abs_dir=None, abs_dif=None, sfc_abs=None):
    bufs = [_buf(abs_dir, ncell, np.float64, "abs_dir", True), _buf(abs_dif, ncell, np.float64, "abs_dif", True),
            _buf(sfc_abs, ncol, np.float64, "sfc_abs", True)]
    mem = _same_mem(*bufs)
    return _check(library().rt_fields_split(h, *[p for p, _ in bufs], mem))


def rt_heating_rate(h, ncell, hr, which=0):
    p, mem = _buf(hr, ncell, np.float64, "hr", True)
    return _check(library().rt_heating_rate(h, p, int(which), mem))


def rt_reset_tallies(h):
    return _check(library().rt_reset_tallies(h))


def rt_stats(h) -> dict:
    s = rt_stats_t()
    _check(library().rt_stats(h, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in rt_stats_t._fields_}


def rt_synchronize(h):
    return _check(library().rt_synchronize(h))


def rt_trace_noalloc(nx, ny, nz, dx, dy, dz, k_gas, ssa_gas, k_cld, ssa_cld, g_cld, albedo, sza_deg,
                     azimuth_deg, toa_flux, photons, seed, abs_dir, abs_dif, sfc_dir, sfc_dif, toa_up,
                     coarse=(0, 0, 0), stream=None) -> int:
    """Trace without any allocation into caller-owned CUDA tensors; returns the event count.

    For callers that may not allocate device memory (see include/rt.h). All
    buffers must be CUDA tensors; outputs are accumulated.
    """
    ncell, ncol = int(nx) * int(ny) * int(nz), int(nx) * int(ny)
    ins = [_buf(a, ncell, np.float32, n) for a, n in
           zip((k_gas, ssa_gas, k_cld, ssa_cld, g_cld), ("k_gas", "ssa_gas", "k_cld", "ssa_cld", "g_cld"))]
    ins.append(_buf(albedo, ncol, np.float32, "albedo"))
    outs = [_buf(abs_dir, ncell, np.float64, "abs_dir", True), _buf(abs_dif, ncell, np.float64, "abs_dif", True)]
    outs += [_buf(a, ncol, np.float64, n, True) for a, n in
             zip((sfc_dir, sfc_dif, toa_up), ("sfc_dir", "sfc_dif", "toa_up"))]
    if _same_mem(*ins, *outs) != RT_DEVICE:
        raise ValueError("rt_trace_noalloc takes device buffers only")
    sptr = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    ev = ctypes.c_uint64(0)
    _check(library().rt_trace_noalloc(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz),
                                      *[p for p, _ in ins], int(coarse[0]), int(coarse[1]), int(coarse[2]),
                                      float(sza_deg), float(azimuth_deg), float(toa_flux), int(photons),
                                      int(seed) & 0xFFFFFFFFFFFFFFFF, *[p for p, _ in outs], sptr,
                                      ctypes.byref(ev)))
    return ev.value


def rt_step_create(h, ncell, ncol, fields, photons, albedo=None, abs3d=None, hr=None, sfc_dir=None,
                   sfc_dif=None, toa_up=None, homogenize=0, optics=None) -> int:
    """Record a coupled-model step over CUDA tensors; returns the step pointer.

    `fields` are the five split optics fields (or four total-optics fields, with
    optics=RT_OPTICS_TOTAL); every buffer must be a CUDA tensor and stay alive
    until rt_step_destroy.
    """
    optics = (RT_OPTICS_SPLIT if len(fields) == 5 else RT_OPTICS_TOTAL) if optics is None else optics
    ins = [_buf(a, ncell, np.float32, "field%d" % q) for q, a in enumerate(fields)]
    ins.append(_buf(albedo, ncol, np.float32, "albedo"))
    outs = [_buf(abs3d, ncell, np.float64, "abs3d", True), _buf(hr, ncell, np.float64, "hr", True)]
    outs += [_buf(a, ncol, np.float64, n, True) for a, n in
             zip((sfc_dir, sfc_dif, toa_up), ("sfc_dir", "sfc_dif", "toa_up"))]
    if _same_mem(*ins, *outs) != RT_DEVICE:
        raise ValueError("rt_step_create takes device buffers only")
    d = rt_step_desc()
    d.optics = int(optics)
    for q, (ptr, _) in enumerate(ins[:-1]):
        d.field[q] = ptr
    d.albedo = ins[-1][0]
    d.photons = int(photons)
    d.abs3d, d.hr, d.sfc_dir, d.sfc_dif, d.toa_up = [ptr for ptr, _ in outs]
    d.homogenize = int(homogenize)
    out = ctypes.c_void_p(0)
    _check(library().rt_step_create(h, ctypes.byref(d), ctypes.byref(out)))
    return out.value


def rt_step_launch(step, sza_deg, azimuth_deg, toa_flux, diffuse_fraction=0.0, seed=1):
    _check(library().rt_step_launch(step, float(sza_deg), float(azimuth_deg), float(toa_flux),
                                    float(diffuse_fraction), int(seed) & 0xFFFFFFFFFFFFFFFF))


def rt_step_destroy(step):
    _check(library().rt_step_destroy(step))


def rt_debug_philox(ctr, key) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    if ctr.shape[0] != key.shape[0]:
        raise ValueError("ctr and key must have the same number of blocks")
    out = np.zeros_like(ctr)
    _check(library().rt_debug_philox(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, ctr.shape[0]))
    return out


def rt_debug_sample(kind: str, n: int, seed: int = 1, g: float = 0.0) -> np.ndarray:
    k = {"rayleigh": 0, "hg": 1, "lambert": 2}[kind]
    out = np.empty(n, dtype=np.float32)
    _check(library().rt_debug_sample(k, float(g), int(n), int(seed), out.ctypes.data))
    return out


def rt_debug_sobol(k0: int, n: int, sx: int = 0, sy: int = 0) -> np.ndarray:
    """(n, 2) uint32 Sobol points k0..k0+n-1 from the device, XORed with (sx, sy)."""
    out = np.empty((n, 2), dtype=np.uint32)
    _check(library().rt_debug_sobol(int(k0), int(n), int(sx), int(sy), out.ctypes.data))
    return out


def rt_probe_read(buf, nbytes: int, reps: int, sink, stream=None):
    """Read nbytes of the device buffer buf reps times (L2-cached 16-byte loads)."""
    sptr = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(library().rt_probe_read(buf.data_ptr(), int(nbytes), int(reps), sink.data_ptr(), sptr))


def rt_debug_turn(d, mu, phi) -> np.ndarray:
    d = np.ascontiguousarray(d, dtype=np.float32)
    mu = np.ascontiguousarray(mu, dtype=np.float32)
    phi = np.ascontiguousarray(phi, dtype=np.float32)
    out = np.empty((mu.size, 3), dtype=np.float32)
    _check(library().rt_debug_turn(d.ctypes.data, mu.ctypes.data, phi.ctypes.data, out.ctypes.data, mu.size))
    return out


# ---- a small object wrapper over one handle ---------------------------------------

class Tracer:
    """One scene handle: grid, optics, surface, acceleration grid and tallies."""

    def __init__(self, nx, ny, nz, dx, dy, dz, stream=None):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dx, self.dy, self.dz = float(dx), float(dy), float(dz)
        self.ncell = self.nx * self.ny * self.nz
        self.ncol = self.nx * self.ny
        self.h = rt_create(nx, ny, nz, dx, dy, dz)
        if stream is not None:
            rt_set_stream(self.h, stream)

    @classmethod
    def from_scene(cls, scene, cx=0, cy=0, cz=0, stream=None, **options):
        t = cls(scene.nx, scene.ny, scene.nz, scene.dx, scene.dy, scene.dz, stream=stream)
        if options:
            t.set_options(**options)
        t.set_optics(*scene.fields())
        t.set_surface(scene.albedo)
        t.build_accel(cx, cy, cz)
        return t

    def close(self):
        if getattr(self, "h", None):
            rt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_options(self, **kw):
        rt_set_options(self.h, **kw)

    def options(self) -> dict:
        return rt_get_options(self.h)

    def set_stream(self, stream):
        rt_set_stream(self.h, stream)

    def set_optics(self, k_gas, ssa_gas, k_cld, ssa_cld, g_cld):
        rt_set_optics(self.h, self.ncell, k_gas, ssa_gas, k_cld, ssa_cld, g_cld)

    def set_surface(self, albedo):
        rt_set_surface(self.h, self.ncol, albedo)

    def build_accel(self, cx=0, cy=0, cz=0):
        rt_build_accel(self.h, cx, cy, cz)

    def trace(self, sza_deg, azimuth_deg, toa_flux, photons, seed, diffuse_fraction=0.0):
        if diffuse_fraction:
            rt_trace_ex(self.h, sza_deg, azimuth_deg, toa_flux, diffuse_fraction, 0, photons, photons, seed)
        else:
            rt_trace(self.h, sza_deg, azimuth_deg, toa_flux, photons, seed)

    def trace_range(self, sza_deg, azimuth_deg, toa_flux, begin, count, total, seed):
        rt_trace_range(self.h, sza_deg, azimuth_deg, toa_flux, begin, count, total, seed)

    def reset(self):
        rt_reset_tallies(self.h)

    def stats(self) -> dict:
        return rt_stats(self.h)

    def synchronize(self):
        rt_synchronize(self.h)

    def fields(self, split: bool = False) -> dict:
        """All output fields as host numpy arrays ([nz][ny][nx] and [ny][nx])."""
        s3, s2 = (self.nz, self.ny, self.nx), (self.ny, self.nx)
        out = {k: np.empty(s3) for k in ("abs3d",)}
        out.update({k: np.empty(s2) for k in ("sfc_dir", "sfc_dif", "toa_up")})
        rt_fields(self.h, self.ncell, self.ncol, out["abs3d"], out["sfc_dir"], out["sfc_dif"], out["toa_up"])
        if split:
            out["abs_dir"], out["abs_dif"] = np.empty(s3), np.empty(s3)
            out["sfc_abs"] = np.empty(s2)
            rt_fields_split(self.h, self.ncell, self.ncol, out["abs_dir"], out["abs_dif"], out["sfc_abs"])
        return out

    def heating_rate(self, which: int = 0) -> np.ndarray:
        hr = np.empty((self.nz, self.ny, self.nx))
        rt_heating_rate(self.h, self.ncell, hr, which)
        return hr
