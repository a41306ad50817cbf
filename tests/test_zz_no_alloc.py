"""The allocation-free entry point gives the same results as the handle API.

sp_mc_simulate_noalloc serves callers that cannot allocate device memory;
it works in a fixed array inside the library.  Here it is called twice in a
row through the C ABI and each result is compared with a handle-based run of
the same mask, optics, photon count and seed in the same tally mode.  Both
run the same kernel on the same photons, so the integer tallies must agree
exactly and the FP64 estimators to rounding.  The second call also shows
that the array's leftover contents from the first call are cleared.
"""
import numpy as np
import pytest

from paper_2604_13929_gb300 import inputs

pytestmark = pytest.mark.gpu

MUS, MUA, G = 0.5, 0.005, 0.7
RAW = ("raw_R", "raw_T", "raw_A", "raw_gated", "raw_lost", "raw_gain", "batch_photons",
       "raw_depth", "raw_hist", "raw_sum_w", "raw_sum_wP", "raw_sum_wP2")
COUNTS = ("launched", "interactions", "scatters", "rr_survive", "rr_kill", "exit_R", "exit_T",
          "gated_n", "steps", "solid_steps")
FLOATS = ("R", "T", "A", "gated", "lost", "gain", "closure", "phi_3d", "phi_1d", "phi_pore",
          "r", "ratio", "porosity", "s_max", "escape_weight", "pore_path_mean")


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_13929_gb300 import build
    build.build()
    from paper_2604_13929_gb300 import spmc
    mask = inputs.spinodal_mask((40, 36, 44), 0.70, 300, seed=3, device="cuda")
    return torch, spmc, mask


def _reference(spmc, mask, n, seed):
    sim = spmc.Simulation(mask, MUS, MUA, G, tally_field=0)
    sim.run(n, seed)
    t = sim.tallies()
    sim.close()
    return t


def _same(a, b):
    for k in RAW:
        assert np.array_equal(a[k], b[k]), k
    for k in COUNTS:
        assert a[k] == b[k], k
    for k in FLOATS:
        assert np.isclose(a[k], b[k], rtol=1e-12, atol=0), k
    assert np.allclose(a["depth"], b["depth"], rtol=1e-12, equal_nan=True)


def test_no_alloc_entry_point_matches_handle_api_twice(setup):
    torch, spmc, mask = setup
    nz, ny, nx = mask.shape
    d_mask = torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    n, seed = 60000, 20260809
    ref = _reference(spmc, mask, n, seed)
    for _ in range(2):
        got = spmc.sp_mc_simulate_noalloc(d_mask, nx, ny, nz, 1.0, MUS, MUA, G, n, seed)
        _same(got, ref)
        assert got["photons"] == n and got["status"] == 0


def test_no_alloc_ragged_sides_after_a_different_volume(setup):
    """Sides that are not multiples of 4 (partial bricks in the packing and
    the voxel counts), called right after a call on a different volume, then
    again: each result equals the handle API's."""
    torch, spmc, mask = setup
    ragged = inputs.spinodal_mask((37, 33, 41), 0.80, 300, seed=4, device="cuda")
    n, seed = 40000, 77
    ref = _reference(spmc, ragged, n, seed)
    d_big = torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    d_rag = torch.from_numpy(np.ascontiguousarray(ragged)).cuda()
    nz, ny, nx = mask.shape
    spmc.sp_mc_simulate_noalloc(d_big, nx, ny, nz, 1.0, MUS, MUA, G, 5000, 1)
    for _ in range(2):
        got = spmc.sp_mc_simulate_noalloc(d_rag, 41, 33, 37, 1.0, MUS, MUA, G, n, seed)
        _same(got, ref)


def test_no_alloc_limit_is_exactly_2_pow_18_bricks(setup):
    """256^3 (exactly 2^18 bricks) is accepted and matches the handle API;
    one more z-layer (65 brick layers) is refused on the host with a buffer
    of the full size behind the pointer."""
    torch, spmc, _ = setup
    mask = inputs.random_mask((256, 256, 256), 0.9, 6)
    n, seed = 20000, 5
    ref = _reference(spmc, mask, n, seed)
    d_mask = torch.from_numpy(mask).cuda()
    got = spmc.sp_mc_simulate_noalloc(d_mask, 256, 256, 256, 1.0, MUS, MUA, G, n, seed)
    _same(got, ref)
    del d_mask
    d_over = torch.zeros((257, 256, 256), dtype=torch.uint8, device="cuda")
    with pytest.raises(spmc.SpmcError) as e:
        spmc.sp_mc_simulate_noalloc(d_over, 256, 256, 257, 1.0, MUS, MUA, G, n, seed)
    assert e.value.code == spmc.SP_EINVAL and "too large" in str(e.value)


def test_no_alloc_entry_point_rejects_oversized_volumes(setup):
    """Volumes above the documented 2^18-brick limit are refused on the host,
    before any device work (the mask pointer is never read)."""
    torch, spmc, mask = setup
    n = 4096
    assert ((n + 3) // 4) ** 3 > 2 ** 18        # far beyond the limit: must be rejected
    d_mask = torch.zeros(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(spmc.SpmcError) as e:
        spmc.sp_mc_simulate_noalloc(d_mask, n, n, n, 1.0, MUS, MUA, G, 10, 1)
    assert e.value.code == spmc.SP_EINVAL and "too large" in str(e.value)
