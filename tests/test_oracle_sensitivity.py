"""How far last-ulp differences in transcendental functions carry along a
history: the reading behind the FP64-transport parity bounds.

The FP64 GPU transport evaluates the oracle's formulas in the oracle's order
(no FMA contraction, IEEE division and square root), so the only arithmetic
difference left is in exp, expm1, log, sin and cos, whose CUDA versions are
accurate to 1-2 ulp while the host libm is (almost always) correctly rounded.
This test gives the oracle itself exactly that kind of difference: a copy of
its source is compiled with each of those five functions moved by -1, 0 or +1
ulp (chosen by a hash of the argument), and the same photons are run through
both builds on a Bernoulli mask with many solid/pore interfaces.

Each interface crossing turns a position difference into an optical-depth
difference, so the tiny perturbations grow along a history.  The observed
rates are the bounds the GPU test uses: >= 99.9 % of photons keep the same
integer event record, while only >= 99.5 % keep every final value (w, P, s,
A) within 1e-6 relative -- 99.9 % would be too tight even for the oracle
against itself.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_13929_gb300 import inputs

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

PERTURB = r'''
#include <math.h>
#include <stdint.h>
#include <string.h>
static double ulp_nudge(double x, double arg) {
    uint64_t b;
    memcpy(&b, &arg, 8);
    b ^= b >> 29; b *= 0xbf58476d1ce4e5b9ull; b ^= b >> 32;
    switch ((int)(b % 3)) {
    case 0: return nextafter(x, -INFINITY);
    case 2: return nextafter(x, INFINITY);
    default: return x;
    }
}
#define exp(a) ulp_nudge(exp(a), (a))
#define expm1(a) ulp_nudge(expm1(a), (a))
#define log(a) ulp_nudge(log(a), (a))
#define sin(a) ulp_nudge(sin(a), (a))
#define cos(a) ulp_nudge(cos(a), (a))
'''


@pytest.fixture(scope="module")
def perturbed(tmp_path_factory):
    src = open(os.path.join(ORACLE_DIR, "spmc_oracle.c")).read()
    anchor = '#include "spmc_oracle.h"'
    assert anchor in src
    d = tmp_path_factory.mktemp("perturbed_oracle")
    c = d / "perturbed.c"
    c.write_text(src.replace(anchor, anchor + "\n" + PERTURB, 1))
    so = d / "libperturbed.so"
    subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", f"-I{ORACLE_DIR}", str(c), "-o", str(so), "-lm"])
    lib = ctypes.CDLL(str(so))
    base = orc.lib()
    for name in ("or_run", "or_default_path_cap"):
        getattr(lib, name).restype = getattr(base, name).restype
        getattr(lib, name).argtypes = getattr(base, name).argtypes
    return lib


def _run(lib, *args, **kw):
    saved = orc._lib
    orc._lib = lib
    try:
        return orc.run(*args, **kw)
    finally:
        orc._lib = saved


def test_ulp_level_differences_bound_whole_history_agreement(perturbed):
    mask = inputs.random_mask((22, 13, 10), 0.55, 9)
    n = 20000
    args = (mask, 0.7, 0.02, 0.6, n, 4242)
    a = orc.run(*args, n_rec=n)
    b = _run(perturbed, *args, n_rec=n)
    same = np.all(a["rec_ints"] == b["rec_ints"], axis=1)
    vclose = np.all(np.isclose(b["rec_vals"], a["rec_vals"], rtol=1e-6, atol=1e-12), axis=1)
    # the perturbation is real: some histories are touched at all
    assert not np.array_equal(a["rec_vals"], b["rec_vals"])
    # the bounds of the FP64 GPU test hold for the oracle against itself ...
    assert same.mean() >= 0.999, same.mean()
    assert vclose.mean() >= 0.995, vclose.mean()
    # ... and the tighter 99.9 % on final values would not
    assert vclose.mean() < 0.999, vclose.mean()
    # aggregate integer counts stay within the GPU test's 0.1 %
    for k in ("interactions", "exit_R", "exit_T", "rr_kill", "steps"):
        assert abs(a["counts"][k] - b["counts"][k]) <= max(2, 1e-3 * a["counts"][k]), k


def test_ulp_level_differences_over_long_histories(perturbed):
    """512^3 tiled spinodal mask, phi = 0.90 (about 1600 voxel steps and 50
    interactions per photon, photon ids above 2^63): the longer histories let
    the same one-ulp differences flip more of them -- about 92 % stay
    identical -- while the first 8 interaction sites all still agree and the
    aggregate counts move by up to about half a percent (within 1 %).  These
    are the bounds of the 512^3 GPU test."""
    tile = inputs.spinodal_mask(64, 0.90, 1000, seed=3, device="cpu")
    mask = np.ascontiguousarray(np.tile(tile, (8, 8, 8)))
    n, pid0 = 10000, 2 ** 63 + 3 * 2 ** 32 - 2 ** 12
    args = (mask, 0.5, 0.005, 0.7, n, 20260809)
    a = orc.run(*args, pid_begin=pid0, n_rec=n, field=False)
    b = _run(perturbed, *args, pid_begin=pid0, n_rec=n, field=False)
    same = np.all(a["rec_ints"] == b["rec_ints"], axis=1)
    first = np.all(np.nan_to_num(np.abs(a["rec_sites"] - b["rec_sites"])) <= 1e-9, axis=(1, 2))
    assert first.mean() >= 0.999, first.mean()
    assert 0.90 <= same.mean() < 0.99, same.mean()
    for k in ("interactions", "exit_R", "exit_T", "rr_kill", "steps", "solid_steps"):
        assert abs(a["counts"][k] - b["counts"][k]) <= max(10, 1e-2 * a["counts"][k]), k
