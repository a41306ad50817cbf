"""Python side of the FP64 CPU oracle (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It compiles ``spmc_oracle.c`` with gcc
into ``oracle/_build`` on first use, runs photons through it, and turns the
integer tallies into the paper's estimators with plain numpy in FP64:

* R, T, A from independent counters (Eq. RTA) and their closure (Eq. closure);
* fluence per unit incident flux, Phi/S0 = F * nx * ny / N, which is
  Eq. Phi_norm for a steady source with the t_end factor dropped;
* the solid-weighted mean <Phi>_3D (Eq. Phi_MC3D), the volume mean <Phi>_1D
  (Eq. Phi_MC1D), the pore mean, the phase contrast r (Eq. r_def), the
  concentration ratio and the dilution identity (Eq. dilution);
* depth profiles per phase (Sec. 3.5(b), App. B post-processing);
* exit-weighted pore-path statistics (Sec. 3.5(c)).
Standard errors come from 16 batch means over photon id modulo 16 (the
replica method of the convergence study, SI S4.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spmc_oracle.c")
_HDR = os.path.join(_HERE, "spmc_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libspmc_oracle.so")

NBATCH, NBIN, NHIST = 16, 64, 257
Q32 = float(2 ** 32)
Q16 = float(2 ** 16)
COUNT_NAMES = ("launched", "interactions", "scatters", "rr_survive", "rr_kill",
               "exit_R", "exit_T", "gated", "steps", "solid_steps")
EXIT_R, EXIT_T, EXIT_RR, EXIT_GATE = 1, 2, 3, 4


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("mask", ctypes.POINTER(ctypes.c_uint8)),
                ("mus", ctypes.c_double), ("mua", ctypes.c_double), ("g", ctypes.c_double),
                ("s_max", ctypes.c_double), ("rr_weight", ctypes.c_double),
                ("rr_mult", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("lateral_bc", ctypes.c_int)]


_U64 = ctypes.c_uint64


class _Tallies(ctypes.Structure):
    _fields_ = [("R", _U64 * NBATCH), ("T", _U64 * NBATCH), ("A", _U64 * NBATCH),
                ("gated", _U64 * NBATCH), ("lost", _U64 * NBATCH), ("gain", _U64 * NBATCH),
                ("photons", _U64 * NBATCH),
                ("depth", _U64 * (NBATCH * 2 * NBIN)),
                ("hist", _U64 * NHIST),
                ("sum_w", _U64 * 2), ("sum_wP", _U64 * 2), ("sum_wP2", _U64 * 2),
                ("counts", _U64 * len(COUNT_NAMES))]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, no fast-math) if stale."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp",
                               "-Wall", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.or_run.restype = ctypes.c_int
            _lib.or_run.argtypes = [ctypes.POINTER(_Problem), _U64, _U64, ctypes.c_int,
                                    ctypes.POINTER(_Tallies), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, _U64]
            _lib.or_uniform.restype = ctypes.c_double
            _lib.or_uniform.argtypes = [ctypes.c_uint32]
            _lib.or_hg_cos.restype = ctypes.c_double
            _lib.or_hg_cos.argtypes = [ctypes.c_double, ctypes.c_double]
            _lib.or_rotate.restype = None
            _lib.or_rotate.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                       ctypes.c_double]
            _lib.or_default_path_cap.restype = ctypes.c_double
            _lib.or_default_path_cap.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_double]
            _lib.or_philox4x32_10.restype = None
            _lib.or_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
        return _lib


# ------------------------------------------------------------ primitives --

def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


def uniform(r: int) -> float:
    return lib().or_uniform(int(r) & 0xFFFFFFFF)


def hg_cos(u: float, g: float) -> float:
    return lib().or_hg_cos(float(u), float(g))


def rotate(d, cost: float, phi: float):
    a = (ctypes.c_double * 3)(*[float(x) for x in d])
    lib().or_rotate(a, float(cost), float(phi))
    return np.array(a[:], dtype=np.float64)


def default_path_cap(nz: int, porosity: float, mus: float, mua: float, g: float) -> float:
    return lib().or_default_path_cap(int(nz), float(porosity), float(mus), float(mua), float(g))


# ------------------------------------------------------------------ run ---

def run(mask: np.ndarray, mus: float, mua: float, g: float, n_photons: int, seed: int,
        s_max: float | None = None, pid_begin: int = 0, rr_weight: float = 1e-4,
        rr_mult: float = 10.0, n_threads: int = 0, field: bool = True, n_rec: int = 0,
        lateral_bc: str = "periodic") -> dict:
    """Run photons [pid_begin, pid_begin + n_photons) through a mask.

    ``mask`` is uint8 (nz, ny, nx), 1 = pore.  ``mus``/``mua`` are the solid
    coefficients times the voxel edge.  ``lateral_bc`` is "periodic" or
    "mirror".  Returns raw integer tallies.
    """
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    nz, ny, nx = mask.shape
    if s_max is None:
        s_max = default_path_cap(nz, float(mask.mean()), mus, mua, g)
    pb = _Problem(nx, ny, nz, mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                  float(mus), float(mua), float(g), float(s_max), float(rr_weight),
                  float(rr_mult), int(seed) & 0xFFFFFFFFFFFFFFFF,
                  {"periodic": 0, "mirror": 1}[lateral_bc])
    t = _Tallies()
    fld = np.zeros(mask.shape, dtype=np.uint64) if field else None
    sites = np.zeros((n_rec, 8, 3)) if n_rec else None
    ints = np.zeros((n_rec, 4), dtype=np.int64) if n_rec else None
    vals = np.zeros((n_rec, 4)) if n_rec else None
    ptr = lambda a: None if a is None else a.ctypes.data  # noqa: E731
    rc = lib().or_run(ctypes.byref(pb), pid_begin, pid_begin + n_photons, int(n_threads),
                      ctypes.byref(t), ptr(fld), ptr(sites), ptr(ints), ptr(vals), n_rec)
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    u = lambda a: np.frombuffer(a, dtype=np.uint64).copy()  # noqa: E731
    out = {
        "mask": mask, "n_photons": int(n_photons), "s_max": float(s_max),
        "R": u(t.R), "T": u(t.T), "A": u(t.A), "gated": u(t.gated), "lost": u(t.lost),
        "gain": u(t.gain), "photons": u(t.photons),
        "depth": u(t.depth).reshape(NBATCH, 2, NBIN), "hist": u(t.hist),
        "sum_w": int(t.sum_w[0]) + (int(t.sum_w[1]) << 64),
        "sum_wP": int(t.sum_wP[0]) + (int(t.sum_wP[1]) << 64),
        "sum_wP2": int(t.sum_wP2[0]) + (int(t.sum_wP2[1]) << 64),
        "counts": {k: int(v) for k, v in zip(COUNT_NAMES, t.counts)},
        "field": fld,
    }
    if n_rec:
        out["rec_sites"], out["rec_ints"], out["rec_vals"] = sites, ints, vals
    return out


# ------------------------------------------------------- normalisation ---

def exact_sum(a: np.ndarray) -> int:
    """Exact integer sum of a uint64 array (split into 32-bit halves)."""
    a = np.asarray(a, dtype=np.uint64).ravel()
    lo = int(np.sum(a & np.uint64(0xFFFFFFFF), dtype=np.uint64))
    hi = int(np.sum(a >> np.uint64(32), dtype=np.uint64))
    return (hi << 32) + lo


def bin_of_layer(nz: int) -> np.ndarray:
    return (np.arange(nz) * NBIN) // nz


def phase_counts(mask: np.ndarray) -> np.ndarray:
    """Voxel count per (phase, depth bin); phase 0 solid, 1 pore."""
    nz = mask.shape[0]
    per_layer_pore = mask.reshape(nz, -1).astype(np.int64).sum(axis=1)
    per_layer_all = np.full(nz, mask.shape[1] * mask.shape[2], dtype=np.int64)
    c = np.zeros((2, NBIN), dtype=np.int64)
    np.add.at(c[1], bin_of_layer(nz), per_layer_pore)
    np.add.at(c[0], bin_of_layer(nz), per_layer_all - per_layer_pore)
    return c


def _mean_se(per_batch_values: np.ndarray):
    v = np.asarray(per_batch_values, dtype=np.float64)
    return float(v.mean(axis=0)) if v.ndim == 1 else v.mean(axis=0), \
        (v.std(axis=0, ddof=1) / np.sqrt(v.shape[0]))


def phase_estimators(phi_3d: float, phi_pore: float, porosity: float) -> dict:
    """Decomposition <Phi>_1D = phi <Phi>_pore + (1 - phi) <Phi>_3D, the
    phase contrast r (Eq. r_def), the concentration ratio <Phi>_3D/<Phi>_1D
    and the dilution prediction 1/[phi r + (1 - phi)] (Eq. dilution)."""
    phi_1d = porosity * phi_pore + (1.0 - porosity) * phi_3d
    r = phi_pore / phi_3d
    inv = porosity * r + (1.0 - porosity)
    return {"phi_1d": phi_1d, "r": r, "ratio": phi_3d / phi_1d,
            "predicted_ratio": 1.0 / inv, "predicted_ratio_inv": inv}


def normalise(res: dict) -> dict:
    """FP64 estimators from the raw tallies of :func:`run`."""
    mask = res["mask"]
    nz, ny, nx = mask.shape
    nb = res["photons"].astype(np.float64)
    N = float(nb.sum())
    out = {"N": N}
    for k in ("R", "T", "A", "gated", "lost", "gain"):
        tot = exact_sum(res[k])
        out[k] = tot / Q32 / N
        per = res[k].astype(np.float64) / Q32 / nb
        out[k + "_se"] = float(per.std(ddof=1) / np.sqrt(NBATCH))
    out["closure"] = out["R"] + out["T"] + out["A"] + out["gated"] + out["lost"] - out["gain"]
    out["RTA"] = out["R"] + out["T"] + out["A"]

    cnt = phase_counts(mask)
    n_pore = int(cnt[1].sum())
    n_vox = nx * ny * nz
    out["porosity"] = n_pore / n_vox
    scale = nx * ny / (N * Q32)

    # phase sums from the direct depth tallies (exact integers)
    dsum = np.zeros((2, NBIN), dtype=object)
    for p in range(2):
        for b in range(NBIN):
            dsum[p, b] = exact_sum(res["depth"][:, p, b])
    tot_solid = sum(dsum[0]) * scale
    tot_pore = sum(dsum[1]) * scale
    n_solid = n_vox - n_pore
    out["phi_3d"] = tot_solid / n_solid if n_solid else float("nan")
    out["phi_pore"] = tot_pore / n_pore if n_pore else float("nan")
    out["phi_1d"] = (tot_solid + tot_pore) / n_vox
    est = phase_estimators(out["phi_3d"], out["phi_pore"], out["porosity"])
    out["r"], out["ratio"] = est["r"], est["ratio"]
    out["identity_residual"] = out["ratio"] * est["predicted_ratio_inv"] - 1.0

    # depth profiles per phase with batch-means SE
    with np.errstate(invalid="ignore", divide="ignore"):
        prof = np.array([[float(dsum[p, b]) for b in range(NBIN)] for p in range(2)]) * scale
        prof = prof / cnt
        per = res["depth"].astype(np.float64) * (nx * ny / Q32) / nb[:, None, None] / cnt[None]
        all_cnt = cnt.sum(axis=0)
        prof_all = (np.array([float(dsum[0, b] + dsum[1, b]) for b in range(NBIN)]) * scale
                    / all_cnt)
        per_all = (res["depth"].astype(np.float64).sum(axis=1) * (nx * ny / Q32)
                   / nb[:, None] / all_cnt[None])
    out["depth"] = prof                     # (2, 64): solid, pore
    out["depth_se"] = per.std(axis=0, ddof=1) / np.sqrt(NBATCH)
    out["depth_all"] = prof_all
    out["depth_all_se"] = per_all.std(axis=0, ddof=1) / np.sqrt(NBATCH)
    out["depth_count"] = cnt

    # exit-weighted pore path (escaping photons only)
    sw = res["sum_w"]
    out["escape_weight"] = sw / Q32 / N
    out["pore_path_mean"] = (res["sum_wP"] / sw) if sw else float("nan")
    out["pore_path_m2"] = (res["sum_wP2"] / Q16) / (sw / Q32) if sw else float("nan")
    h = res["hist"].astype(np.float64)
    out["pore_path_hist"] = h / Q32 / N
    # P_w(pore path > L): bins of width 4L/256 put L on the edge of bin 64
    out["p_pore_gt_L"] = float(h[64:].sum() / h.sum()) if h.sum() > 0 else float("nan")

    if res.get("field") is not None:
        out["fluence"] = res["field"].astype(np.float64) * scale
    out["counts"] = dict(res["counts"])
    return out


def field_phase_sums(field: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """Exact integer sums of a Q32.32 voxel field per (phase, depth bin)."""
    nz = mask.shape[0]
    bins = bin_of_layer(nz)
    s = np.zeros((2, NBIN), dtype=object)
    for z in range(nz):
        layer = field[z]
        m = mask[z] != 0
        s[1, bins[z]] += exact_sum(layer[m])
        s[0, bins[z]] += exact_sum(layer[~m])
    return s
