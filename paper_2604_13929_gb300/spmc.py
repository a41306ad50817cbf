"""Thin ctypes binding of libspmc (argument marshalling only).

Every step of the Monte Carlo runs in the CUDA library; this module only
converts arguments.  There is no CPU fallback: if ``libspmc.so`` has not been
built, :func:`load` raises, and without a GPU every call that needs one
returns ``SP_ECUDA``, which the wrappers raise as :class:`SpmcError`.

The module-level functions carry the C names (``sp_mc_create``,
``sp_mc_run``, ``sp_mc_tallies``, ...); :class:`Simulation` is a small
convenience owner of one handle.  Streams: ``None`` selects torch's current
CUDA stream when torch has CUDA, else the legacy default stream; a
``torch.cuda.Stream`` or a raw ``cudaStream_t`` integer is passed through.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libspmc.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "spmc.h")

SP_OK, SP_EINVAL, SP_ENOMEM, SP_ECUDA, SP_ESTEPLIMIT, SP_EOVERFLOW = 0, -1, -2, -3, -4, -5
NBATCH, NBIN, NHIST = 16, 64, 257
OPT = {"path_cap": 1, "rr_weight": 2, "rr_mult": 3, "tally_field": 4, "precision": 5,
       "records": 6, "blocks": 7, "threads": 8, "iter_limit": 9, "smem_bricks": 10,
       "pid_offset": 11, "compact": 12, "graph": 13, "lateral_bc": 14, "batch_mode": 15,
       "kernel": 16, "steps_per_pass": 17, "batch_chunk": 18}
ERR_NAMES = {SP_EINVAL: "SP_EINVAL", SP_ENOMEM: "SP_ENOMEM", SP_ECUDA: "SP_ECUDA",
             SP_ESTEPLIMIT: "SP_ESTEPLIMIT", SP_EOVERFLOW: "SP_EOVERFLOW"}

_D, _U64, _I32 = ctypes.c_double, ctypes.c_uint64, ctypes.c_int32


class Result(ctypes.Structure):
    """Mirror of sp_mc_result_t (layout checked against sp_mc_result_size)."""
    _fields_ = [
        ("photons", _U64), ("status", _I32), ("precision", _I32),
        ("s_max", _D), ("porosity", _D),
        ("R", _D), ("T", _D), ("A", _D), ("gated", _D), ("lost", _D), ("gain", _D),
        ("closure", _D), ("R_se", _D), ("T_se", _D), ("A_se", _D),
        ("phi_3d", _D), ("phi_1d", _D), ("phi_pore", _D), ("r", _D), ("ratio", _D),
        ("identity_residual", _D),
        ("depth", _D * (3 * NBIN)), ("depth_count", _U64 * (2 * NBIN)),
        ("escape_weight", _D), ("pore_path_mean", _D), ("pore_path_m2", _D),
        ("p_pore_gt_L", _D), ("pore_hist", _D * NHIST),
        ("launched", _U64), ("interactions", _U64), ("scatters", _U64),
        ("rr_survive", _U64), ("rr_kill", _U64), ("exit_R", _U64), ("exit_T", _U64),
        ("gated_n", _U64), ("steps", _U64), ("solid_steps", _U64),
        ("raw_R", _U64 * NBATCH), ("raw_T", _U64 * NBATCH), ("raw_A", _U64 * NBATCH),
        ("raw_gated", _U64 * NBATCH), ("raw_lost", _U64 * NBATCH), ("raw_gain", _U64 * NBATCH),
        ("batch_photons", _U64 * NBATCH),
        ("raw_depth", _U64 * (2 * NBIN * 2)), ("raw_hist", _U64 * NHIST),
        ("raw_sum_w", _U64 * 2), ("raw_sum_wP", _U64 * 2), ("raw_sum_wP2", _U64 * 2),
    ]

    def to_dict(self) -> dict:
        out = {}
        for name, ctype in self._fields_:
            v = getattr(self, name)
            if hasattr(ctype, "_length_"):
                dt = np.float64 if ctype._type_ is _D else np.uint64
                v = np.ctypeslib.as_array(v).astype(dt).copy()
            out[name] = v
        out["depth"] = out["depth"].reshape(3, NBIN)
        out["depth_count"] = out["depth_count"].reshape(2, NBIN)
        out["raw_depth"] = out["raw_depth"].reshape(2, NBIN, 2)
        return out


class SpmcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def declared_functions() -> list[str]:
    """Names of the functions declared in include/spmc.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(sp_mc_\w+)\s*\(", text)))


def load() -> ctypes.CDLL:
    """Load the in-tree libspmc.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2604_13929_gb300.build` (needs nvcc)")
        lib = ctypes.CDLL(LIB_PATH)
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        sig = {
            "sp_mc_create": (vp, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]),
            "sp_mc_set_option": (ctypes.c_int, [vp, ctypes.c_int, _D]),
            "sp_mc_get_option": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(_D)]),
            "sp_mc_run": (ctypes.c_int, [vp, _U64, _U64, vp]),
            "sp_mc_tallies": (ctypes.c_int, [vp, ctypes.POINTER(Result), vp]),
            "sp_mc_fluence": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, vp]),
            "sp_mc_raw_field": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
            "sp_mc_records": (ctypes.c_int, [vp, _U64, vp, vp, vp, vp]),
            "sp_mc_reset": (ctypes.c_int, [vp, vp]),
            "sp_mc_checkpoint_size": (sz, [vp]),
            "sp_mc_checkpoint": (ctypes.c_int, [vp, vp, sz, vp]),
            "sp_mc_restore": (ctypes.c_int, [vp, vp, sz, vp]),
            "sp_mc_destroy": (None, [vp]),
            "sp_mc_last_error": (ctypes.c_char_p, []),
            "sp_mc_version": (ctypes.c_char_p, []),
            "sp_mc_result_size": (sz, []),
            "sp_mc_batch_create": (vp, [ctypes.c_int, vp, vp, vp]),
            "sp_mc_batch_set_option": (ctypes.c_int, [vp, ctypes.c_int, _D]),
            "sp_mc_batch_get_option": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(_D)]),
            "sp_mc_batch_run": (ctypes.c_int, [vp, vp, _U64, vp]),
            "sp_mc_batch_tallies": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(Result), vp]),
            "sp_mc_batch_raw_field": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, vp]),
            "sp_mc_batch_reset": (ctypes.c_int, [vp, vp]),
            "sp_mc_batch_autotune": (ctypes.c_int, [vp, vp, _U64, ctypes.POINTER(_D), vp]),
            "sp_mc_batch_destroy": (None, [vp]),
            "sp_mc_probe_step_ceiling": (ctypes.c_int, [ctypes.c_int, ctypes.c_int,
                                                        ctypes.c_longlong,
                                                        ctypes.POINTER(_D), ctypes.POINTER(_D)]),
            "sp_mc_simulate_noalloc": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                      _D, _D, _D, _D, _U64, _U64,
                                                      ctypes.POINTER(Result), vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        if lib.sp_mc_result_size() != ctypes.sizeof(Result):
            raise OSError("sp_mc_result_t layout mismatch between library and binding")
        _lib = lib
        return lib


def _check(rc: int):
    if rc != SP_OK:
        raise SpmcError(rc, load().sp_mc_last_error().decode())
    return rc


def stream_handle(stream=None) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _ptr(buf):
    """(address, on_device) of a numpy array or torch tensor."""
    if isinstance(buf, np.ndarray):
        return buf.ctypes.data, 0
    return int(buf.data_ptr()), 1 if buf.is_cuda else 0


# ------------------------------------------------- C-named entry points --

def sp_mc_create(mask, nx: int, ny: int, nz: int, voxel_h: float, mu_s: float, mu_a: float,
                 g: float) -> int:
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if m.size != nx * ny * nz:
        raise ValueError("mask size does not match nx*ny*nz")
    h = load().sp_mc_create(m.ctypes.data, nx, ny, nz, voxel_h, mu_s, mu_a, g)
    if not h:
        msg = load().sp_mc_last_error().decode()
        code = SP_ECUDA if "CUDA" in msg or "device" in msg else SP_EINVAL
        raise SpmcError(code, msg)
    return h


def sp_mc_set_option(h: int, key, value: float):
    _check(load().sp_mc_set_option(h, OPT.get(key, key), float(value)))


def sp_mc_get_option(h: int, key) -> float:
    v = _D()
    _check(load().sp_mc_get_option(h, OPT.get(key, key), ctypes.byref(v)))
    return v.value


def sp_mc_run(h: int, n_photons: int, seed: int, stream=None):
    _check(load().sp_mc_run(h, int(n_photons), int(seed) & (2 ** 64 - 1), stream_handle(stream)))


def sp_mc_tallies(h: int, stream=None, check: bool = True) -> dict:
    r = Result()
    rc = load().sp_mc_tallies(h, ctypes.byref(r), stream_handle(stream))
    if check:
        _check(rc)
    return r.to_dict()


def _float_code(buf) -> int:
    """0 for float64, 1 for float32 (numpy array or torch tensor)."""
    name = str(buf.dtype).replace("torch.", "")
    if name not in ("float64", "float32"):
        raise TypeError("fluence buffer must be float64 or float32")
    return 0 if name == "float64" else 1


def sp_mc_fluence(h: int, dst, stream=None):
    """dst: contiguous float64/float32 numpy array or torch tensor (host or CUDA)."""
    dtype = _float_code(dst)
    addr, dev = _ptr(dst)
    _check(load().sp_mc_fluence(h, addr, dtype, dev, stream_handle(stream)))
    return dst


def sp_mc_raw_field(h: int, dst, stream=None):
    addr, dev = _ptr(dst)
    _check(load().sp_mc_raw_field(h, addr, dev, stream_handle(stream)))
    return dst


def sp_mc_records(h: int, n: int, stream=None):
    sites = np.empty((n, 8, 3))
    ints = np.empty((n, 4), dtype=np.int64)
    vals = np.empty((n, 4))
    _check(load().sp_mc_records(h, n, sites.ctypes.data, ints.ctypes.data, vals.ctypes.data,
                                stream_handle(stream)))
    return sites, ints, vals


def sp_mc_reset(h: int, stream=None):
    _check(load().sp_mc_reset(h, stream_handle(stream)))


def sp_mc_checkpoint_size(h: int) -> int:
    return load().sp_mc_checkpoint_size(h)


def sp_mc_checkpoint(h: int, stream=None) -> bytes:
    n = sp_mc_checkpoint_size(h)
    buf = ctypes.create_string_buffer(n)
    _check(load().sp_mc_checkpoint(h, buf, n, stream_handle(stream)))
    return buf.raw


def sp_mc_restore(h: int, data: bytes, stream=None):
    buf = ctypes.create_string_buffer(data, len(data))
    _check(load().sp_mc_restore(h, buf, len(data), stream_handle(stream)))


def sp_mc_destroy(h: int):
    if h:
        load().sp_mc_destroy(h)


def sp_mc_last_error() -> str:
    return load().sp_mc_last_error().decode()


def sp_mc_version() -> str:
    return load().sp_mc_version().decode()


def sp_mc_probe_step_ceiling(n: int, red: bool, steps_per_thread: int = 20000) -> dict:
    """Measured stepping ceiling (steps/s) of the transport's memory pattern
    through an n^3 volume (n a multiple of 4)."""
    ms, rate = _D(), _D()
    _check(load().sp_mc_probe_step_ceiling(int(n), 1 if red else 0, int(steps_per_thread),
                                           ctypes.byref(ms), ctypes.byref(rate)))
    return {"ms": ms.value, "steps_per_s": rate.value}


def sp_mc_simulate_noalloc(d_mask, nx: int, ny: int, nz: int, voxel_h: float, mu_s: float,
                           mu_a: float, g: float, n_photons: int, seed: int, stream=None) -> dict:
    """One complete simulation through the allocation-free entry point.

    ``d_mask`` is a CUDA uint8 tensor (or a raw device address) holding the
    nz*ny*nx mask, x fastest.  Nothing is allocated on the device, by the
    library or here; the result struct lives in host memory.
    """
    addr = d_mask if isinstance(d_mask, int) else int(d_mask.data_ptr())
    r = Result()
    _check(load().sp_mc_simulate_noalloc(addr, nx, ny, nz, voxel_h, mu_s, mu_a, g,
                                         int(n_photons), int(seed) & (2 ** 64 - 1),
                                         ctypes.byref(r), stream_handle(stream)))
    return r.to_dict()


# ------------------------------------------------------------ convenience --

class Batch:
    """Many masks (uneven sizes, per-problem optics) in one persistent launch.

    ``problems`` is a list of (mask, mu_s, mu_a, g) or (mask, mu_s, mu_a, g,
    voxel_h); masks are uint8 (nz, ny, nx), 1 = pore.
    """

    def __init__(self, problems, **options):
        self.masks = [np.ascontiguousarray(pr[0], dtype=np.uint8) for pr in problems]
        self.n = len(self.masks)
        ptrs = (ctypes.c_void_p * self.n)(*[m.ctypes.data for m in self.masks])
        dims = np.array([[m.shape[2], m.shape[1], m.shape[0]] for m in self.masks],
                        dtype=np.int32)
        optics = np.array([[pr[4] if len(pr) > 4 else 1.0, pr[1], pr[2], pr[3]]
                           for pr in problems], dtype=np.float64)
        self.handle = load().sp_mc_batch_create(self.n, ptrs, dims.ctypes.data,
                                                optics.ctypes.data)
        if not self.handle:
            raise SpmcError(SP_EINVAL, load().sp_mc_last_error().decode())
        for k, v in options.items():
            self.set_option(k, v)

    def set_option(self, key, value):
        _check(load().sp_mc_batch_set_option(self.handle, OPT.get(key, key), float(value)))

    def get_option(self, key) -> float:
        v = _D()
        _check(load().sp_mc_batch_get_option(self.handle, OPT.get(key, key), ctypes.byref(v)))
        return v.value

    def _counts(self, n_photons):
        n = np.broadcast_to(np.asarray(n_photons, dtype=np.uint64), (self.n,))
        return np.ascontiguousarray(n)

    def run(self, n_photons, seed: int, stream=None):
        n = self._counts(n_photons)
        _check(load().sp_mc_batch_run(self.handle, n.ctypes.data, int(seed) & (2 ** 64 - 1),
                                      stream_handle(stream)))
        return self

    def tallies(self, i: int, stream=None) -> dict:
        r = Result()
        _check(load().sp_mc_batch_tallies(self.handle, int(i), ctypes.byref(r),
                                          stream_handle(stream)))
        return r.to_dict()

    def raw_field(self, i: int, stream=None):
        out = np.empty(self.masks[i].shape, dtype=np.uint64)
        _check(load().sp_mc_batch_raw_field(self.handle, int(i), out.ctypes.data, 0,
                                            stream_handle(stream)))
        return out

    def raw_field_to(self, i: int, dst, stream=None):
        """Copy problem i's Q32.32 field into a device buffer (torch uint64/int64 tensor)."""
        assert dst.numel() == self.masks[i].size and dst.element_size() == 8 and dst.is_cuda
        _check(load().sp_mc_batch_raw_field(self.handle, int(i), dst.data_ptr(), 1, stream_handle(stream)))

    def reset(self, stream=None):
        _check(load().sp_mc_batch_reset(self.handle, stream_handle(stream)))

    def autotune(self, n_photons, seed: int, stream=None) -> float:
        n = self._counts(n_photons)
        rate = _D()
        _check(load().sp_mc_batch_autotune(self.handle, n.ctypes.data, int(seed) & (2 ** 64 - 1),
                                           ctypes.byref(rate), stream_handle(stream)))
        return rate.value

    def close(self):
        if getattr(self, "handle", None):
            load().sp_mc_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """Owner of one sp_mc handle.

    ``mask`` is uint8 (nz, ny, nx), 1 = pore.  ``mu_s``/``mu_a`` are in the
    inverse length unit of ``voxel_h`` (use voxel_h = 1 for per-voxel optics).
    """

    def __init__(self, mask, mu_s: float, mu_a: float, g: float, voxel_h: float = 1.0,
                 **options):
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        self.shape = m.shape
        nz, ny, nx = m.shape
        self.handle = sp_mc_create(m, nx, ny, nz, voxel_h, mu_s, mu_a, g)
        for k, v in options.items():
            self.set_option(k, v)

    def set_option(self, key, value):
        sp_mc_set_option(self.handle, key, value)

    def get_option(self, key) -> float:
        return sp_mc_get_option(self.handle, key)

    def run(self, n_photons: int, seed: int, stream=None):
        sp_mc_run(self.handle, n_photons, seed, stream)
        return self

    def tallies(self, stream=None, check: bool = True) -> dict:
        return sp_mc_tallies(self.handle, stream, check)

    def fluence(self, out=None, stream=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        return sp_mc_fluence(self.handle, out, stream)

    def raw_field(self, out=None, stream=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.uint64)
        return sp_mc_raw_field(self.handle, out, stream)

    def records(self, n: int, stream=None):
        return sp_mc_records(self.handle, n, stream)

    def reset(self, stream=None):
        sp_mc_reset(self.handle, stream)

    def checkpoint(self, stream=None) -> bytes:
        return sp_mc_checkpoint(self.handle, stream)

    def restore(self, data: bytes, stream=None):
        sp_mc_restore(self.handle, data, stream)

    def close(self):
        if getattr(self, "handle", None):
            sp_mc_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
