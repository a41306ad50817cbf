"""GPU parity of the fluence surrogate (libspnn) against the FP64 oracle.

Every GPU layer reads BF16 operands and accumulates in FP32 on the tensor
cores; the oracle evaluates the same definition in FP64 on the same
BF16-valued inputs.  Bound per output element, derived from the arithmetic:
FP32 accumulation of K products contributes at most ~K 2^-24 sum|x w| (2^-12
sum|x w| covers K <= 4096 with margin), and a BF16 result adds half an ulp,
2^-9 |y| (2^-8 used).  sum|x w| is the same layer applied to |x| and |w|.
"""
import numpy as np
import pytest
import torch

from oracle import unet_oracle as U
from paper_2604_13929_gb300 import spnn as SP

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2604_13929_gb300 import spnn
    spnn.load()
    return spnn


def bf(a):
    """(B, D, H, W, C) values -> BF16 activation in chunk planes on the GPU."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().to(torch.bfloat16)
    return SP.to_planes(t)


def f64(t):
    """GPU tensor -> float64 numpy; chunk-plane activations come back as (B, D, H, W, C)."""
    if t.dim() == 6:
        t = SP.from_planes(t)
    return t.float().cpu().numpy().astype(np.float64)


def zeros_act(B, D, H, W, C):
    return SP.planes_empty(B, D, H, W, C)


def w_bf(w):
    """Master FP32 weights as the BF16 values the packed operands hold."""
    return torch.from_numpy(w.astype(np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def check(gpu, ref, absref, out_bf16=True, what=""):
    tol = (2.0 ** -8 * np.abs(ref) if out_bf16 else 0.0) + 2.0 ** -12 * absref + 1e-6
    bad = np.abs(gpu - ref) > tol
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(gpu - ref) - tol)))


def rnd(rng, shape, scale=1.0):
    return rng.standard_normal(shape) * scale


def packed(S, kind, cin, cout, which, w):
    wt = torch.from_numpy(w.astype(np.float32)).cuda()
    pk = torch.empty(S.spnn_packed_elems(kind, cin, cout), dtype=torch.bfloat16, device="cuda")
    S.spnn_pack_weights(kind, cin, cout, which, wt, pk)
    return pk


# ------------------------------------------------------------------ forward --

def test_conv3_forward_concat_bias_relu(S):
    rng = np.random.default_rng(1)
    B, D, H, W, c0, c1, co = 2, 4, 8, 16, 16, 32, 48
    x0, x1 = bf(rnd(rng, (B, D, H, W, c0))), bf(rnd(rng, (B, D, H, W, c1)))
    w = rnd(rng, (27, c0 + c1, co), 0.1)
    b = rnd(rng, co, 0.5)
    y = zeros_act(B, D, H, W, co)
    S.spnn_layer_forward(S.CONV3, (B, D, H, W), x0, x1, packed(S, 0, c0 + c1, co, 0, w),
                         torch.tensor(b, dtype=torch.float32, device="cuda"), co, True, y)
    S.spnn_status()
    xin = np.concatenate([f64(x0), f64(x1)], axis=-1)
    ref = U.relu(U.conv3(xin, w_bf(w), b))
    absref = U.conv3(np.abs(xin), np.abs(w_bf(w)), np.abs(b))
    check(f64(y), ref, absref, what="conv3")


def test_conv3_fused_head(S):
    rng = np.random.default_rng(2)
    B, D, H, W, c0, co = 1, 8, 8, 8, 32, 32
    x = bf(rnd(rng, (B, D, H, W, c0)))
    w = rnd(rng, (27, c0, co), 0.1)
    hw = rnd(rng, co)
    y = zeros_act(B, D, H, W, co)
    out = torch.zeros((B, D, H, W), dtype=torch.float32, device="cuda")
    hwt = torch.tensor(hw, dtype=torch.float32, device="cuda")
    hb = torch.tensor([0.25], dtype=torch.float32, device="cuda")
    S.spnn_layer_forward(S.CONV3, (B, D, H, W), x, None, packed(S, 0, c0, co, 0, w), None, co, True, y,
                         head_w=hwt, head_b=hb, head_out=out)
    S.spnn_status()
    yg = f64(y)
    check(yg, U.relu(U.conv3(f64(x), w_bf(w))), U.conv3(np.abs(f64(x)), np.abs(w_bf(w))), what="conv3")
    ref = yg @ hwt.cpu().double().numpy() + 0.25
    tol = 1e-5 * (np.abs(yg) @ np.abs(hw) + 1)
    assert np.all(np.abs(out.cpu().numpy() - ref) <= tol)


def test_down_forward(S):
    rng = np.random.default_rng(3)
    B, D, H, W, c0, co = 2, 8, 8, 16, 32, 64
    x = bf(rnd(rng, (B, D, H, W, c0)))
    w = rnd(rng, (8, c0, co), 0.2)
    b = rnd(rng, co, 0.5)
    y = zeros_act(B, D // 2, H // 2, W // 2, co)
    S.spnn_layer_forward(S.DOWN, (B, D, H, W), x, None, packed(S, 1, c0, co, 0, w),
                         torch.tensor(b, dtype=torch.float32, device="cuda"), co, True, y)
    S.spnn_status()
    check(f64(y), U.relu(U.down(f64(x), w_bf(w), b)), U.down(np.abs(f64(x)), np.abs(w_bf(w)), np.abs(b)),
          what="down")


def test_up_forward_column_tiles(S):
    rng = np.random.default_rng(4)
    B, D, H, W, c0, co = 2, 4, 4, 8, 32, 64       # N = 8 * 64 = 512: four 128-column tiles
    x = bf(rnd(rng, (B, D, H, W, c0)))
    w = rnd(rng, (8, c0, co), 0.2)
    b = rnd(rng, co, 0.5)
    y = zeros_act(B, 2 * D, 2 * H, 2 * W, co)
    S.spnn_layer_forward(S.UP, (B, D, H, W), x, None, packed(S, 2, c0, co, 0, w),
                         torch.tensor(b, dtype=torch.float32, device="cuda"), co, False, y)
    S.spnn_status()
    check(f64(y), U.up(f64(x), w_bf(w), b), U.up(np.abs(f64(x)), np.abs(w_bf(w)), np.abs(b)), what="up")


# ---------------------------------------------------------- input gradient --

def test_conv3_dgrad_split_mask_addend(S):
    rng = np.random.default_rng(5)
    B, D, H, W, c0, c1, co = 2, 4, 8, 16, 16, 32, 48
    dy = bf(rnd(rng, (B, D, H, W, co)))
    w = rnd(rng, (27, c0 + c1, co), 0.1)
    mask0 = bf(rnd(rng, (B, D, H, W, c0)))
    add1 = bf(rnd(rng, (B, D, H, W, c1)))
    dx0 = zeros_act(B, D, H, W, c0)
    dx1 = zeros_act(B, D, H, W, c1)
    S.spnn_layer_dgrad(S.CONV3, (B, D, H, W), dy, packed(S, 0, c0 + c1, co, 1, w), c0, c1, dx0, mask0=mask0,
                       dx1=dx1, addend1=add1)
    S.spnn_status()
    g = U.conv3_dgrad(f64(dy), w_bf(w))
    ga = U.conv3_dgrad(np.abs(f64(dy)), np.abs(w_bf(w)))
    check(f64(dx0), g[..., :c0] * (f64(mask0) > 0), ga[..., :c0], what="dx0")
    check(f64(dx1), g[..., c0:] + f64(add1), ga[..., c0:] + np.abs(f64(add1)), what="dx1")


def test_down_dgrad_scatter(S):
    rng = np.random.default_rng(6)
    B, D, H, W, c0, co = 2, 8, 8, 16, 32, 64       # N = 8 * 32 = 256
    dy = bf(rnd(rng, (B, D // 2, H // 2, W // 2, co)))
    w = rnd(rng, (8, c0, co), 0.2)
    add = bf(rnd(rng, (B, D, H, W, c0)))
    mask = bf(rnd(rng, (B, D, H, W, c0)))
    dx = zeros_act(B, D, H, W, c0)
    S.spnn_layer_dgrad(S.DOWN, (B, D, H, W), dy, packed(S, 1, c0, co, 1, w), c0, 0, dx, addend0=add, mask0=mask)
    S.spnn_status()
    ref = (U.down_dgrad(f64(dy), w_bf(w)) + f64(add)) * (f64(mask) > 0)
    absref = U.down_dgrad(np.abs(f64(dy)), np.abs(w_bf(w))) + np.abs(f64(add))
    check(f64(dx), ref, absref, what="down dgrad")


def test_up_dgrad_gather(S):
    rng = np.random.default_rng(7)
    B, D, H, W, c0, co = 2, 4, 4, 8, 32, 64
    dy = bf(rnd(rng, (B, 2 * D, 2 * H, 2 * W, co)))
    w = rnd(rng, (8, c0, co), 0.2)
    dx = zeros_act(B, D, H, W, c0)
    S.spnn_layer_dgrad(S.UP, (B, D, H, W), dy, packed(S, 2, c0, co, 1, w), c0, 0, dx)
    S.spnn_status()
    check(f64(dx), U.up_dgrad(f64(dy), w_bf(w)), U.up_dgrad(np.abs(f64(dy)), np.abs(w_bf(w))), what="up dgrad")


# --------------------------------------------------------- weight gradient --

@pytest.mark.parametrize("kind", ["conv3", "conv3_concat", "down", "up"])
def test_wgrad(S, kind):
    rng = np.random.default_rng(8)
    B, D, H, W = 2, 8, 8, 16
    if kind.startswith("conv3"):
        c0, c1, co = (16, 32, 48) if kind == "conv3_concat" else (32, 0, 64)
        x0 = bf(rnd(rng, (B, D, H, W, c0)))
        x1 = bf(rnd(rng, (B, D, H, W, c1))) if c1 else None
        dy = bf(rnd(rng, (B, D, H, W, co)))
        xin = f64(x0) if x1 is None else np.concatenate([f64(x0), f64(x1)], axis=-1)
        ref_w, ref_b = U.conv3_wgrad(xin, f64(dy))
        abs_w, abs_b = U.conv3_wgrad(np.abs(xin), np.abs(f64(dy)))
        taps, k = 27, S.CONV3
    elif kind == "down":
        c0, c1, co = 32, 0, 64
        x0, x1 = bf(rnd(rng, (B, D, H, W, c0))), None
        dy = bf(rnd(rng, (B, D // 2, H // 2, W // 2, co)))
        ref_w, ref_b = U.down_wgrad(f64(x0), f64(dy))
        abs_w, abs_b = U.down_wgrad(np.abs(f64(x0)), np.abs(f64(dy)))
        taps, k = 8, S.DOWN
    else:
        c0, c1, co = 32, 0, 64
        D, H, W = 4, 4, 8
        x0, x1 = bf(rnd(rng, (B, D, H, W, c0))), None
        dy = bf(rnd(rng, (B, 2 * D, 2 * H, 2 * W, co)))
        ref_w, ref_b = U.up_wgrad(f64(x0), f64(dy))
        abs_w, abs_b = U.up_wgrad(np.abs(f64(x0)), np.abs(f64(dy)))
        taps, k = 8, S.UP
    dw = torch.zeros((taps, c0 + c1, co), dtype=torch.float32, device="cuda")
    db = torch.zeros(co, dtype=torch.float32, device="cuda")
    S.spnn_layer_wgrad(k, (B, D, H, W), x0, x1, dy, dw, db)
    S.spnn_status()
    check(dw.cpu().numpy().astype(np.float64), ref_w, abs_w, out_bf16=False, what="dw")
    check(db.cpu().numpy().astype(np.float64), ref_b, abs_b, out_bf16=False, what="db")


# -------------------------------------------------------------------- data --

def test_pack_input_log_fluence_profiles(S):
    rng = np.random.default_rng(9)
    B, D, H, W = 3, 8, 4, 8
    mask = (rng.random((B, D, H, W)) < 0.6).astype(np.uint8)
    optics = np.array([[0.5, 0.005, 0.7], [1.9, 0.04, 0.0], [0.11, 0.0012, 0.89]], dtype=np.float32)
    x = zeros_act(B, D, H, W, 16)
    S.spnn_pack_input(torch.from_numpy(mask).cuda(), torch.from_numpy(optics).cuda(), x)
    ref = U.pack_input(mask, optics[:, 0].astype(np.float64), optics[:, 1].astype(np.float64),
                       optics[:, 2].astype(np.float64))
    np.testing.assert_allclose(f64(x), ref, rtol=2.0 ** -7, atol=1e-7)
    raw = rng.integers(0, 2 ** 44, size=(B, D, H, W), dtype=np.uint64)
    raw[0, 0, 0, :4] = 0
    n = np.array([1e6, 3e7, 12345.0])
    out = torch.zeros((B, D, H, W), dtype=torch.float32, device="cuda")
    S.spnn_log_fluence(torch.from_numpy(raw.view(np.int64)).cuda(), torch.from_numpy(n).cuda(), out, floor=1e-6)
    S.spnn_status()
    ref = np.stack([U.log_fluence(raw[b], W, H, int(n[b])) for b in range(B)])
    assert np.all(np.abs(out.cpu().numpy() - ref) <= 2e-6 * (1 + np.abs(ref)))
    prof = torch.zeros((B, 2, D), dtype=torch.float32, device="cuda")
    S.spnn_phase_profiles(out, torch.from_numpy(mask).cuda(), prof)
    S.spnn_status()
    pref = U.phase_profiles(out.cpu().numpy().astype(np.float64), mask)
    np.testing.assert_allclose(prof.cpu().numpy(), pref, rtol=2e-6, equal_nan=True)


# ----------------------------------------------------------------- network --

C0, N, BATCH = 16, 16, 16


@pytest.fixture(scope="module")
def net_run(S):
    """One forward and backward of the c0 = 16 U-Net on 16 cubes of 16^3."""
    rng = np.random.default_rng(10)
    params = U.init_params(C0, 21)
    flat = S.flatten_params(params, C0)
    net = S.UNet(C0, N, BATCH)
    assert net.param_count == flat.size
    net.set_params(flat)
    mask = (rng.random((BATCH, N, N, N)) < 0.7).astype(np.uint8)
    optics = np.stack([rng.uniform(0.1, 2.0, BATCH), rng.uniform(0.001, 0.05, BATCH),
                       rng.uniform(0.0, 0.9, BATCH)], axis=1).astype(np.float32)
    x = zeros_act(BATCH, N, N, N, 16)
    S.spnn_pack_input(torch.from_numpy(mask).cuda(), torch.from_numpy(optics).cuda(), x)
    pred = torch.zeros((BATCH, N, N, N), dtype=torch.float32, device="cuda")
    net.forward(x, pred)
    acts = [net.activation(i, BATCH) for i in range(20)]
    target = torch.from_numpy(rng.standard_normal((BATCH, N, N, N)).astype(np.float32) * 0.3).cuda()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.backward(target, loss)
    S.spnn_status()
    grads = net.get_grads()
    yield dict(net=net, params=params, flat=flat, x=x, pred=pred, acts=acts, target=target, loss=loss,
               grads=grads, mask=mask)
    net.close()


def _layer_inputs(run):
    table = U.layer_table(C0)
    act = {"x": f64(run["x"])}
    for (name, *_), a in zip(table, run["acts"]):
        act[name] = f64(a)
    return table, act


def test_unet_forward_layerwise(S, net_run):
    """Each layer's GPU output against the oracle layer applied to the GPU's
    own BF16 inputs: checks the wiring (sources, concatenation order, strides,
    activations) layer by layer at the tight per-layer bound."""
    table, act = _layer_inputs(net_run)
    params = net_run["params"]
    prev = "x"
    for name, kind, _, _, relu in table:
        w, b = params[name]
        srcs = U.SKIP_OF.get(name, (prev,))
        xin = np.concatenate([act[s] for s in srcs], axis=-1)
        op = {"conv3": U.conv3, "down": U.down, "up": U.up}[kind]
        ref = op(xin, w_bf(w), b)
        absref = op(np.abs(xin), np.abs(w_bf(w)), np.abs(b))
        check(act[name], U.relu(ref) if relu else ref, absref, what=name)
        prev = name
    hw, hb = params["head"]
    ref = act["c0b"] @ hw.astype(np.float32).astype(np.float64) + float(np.float32(hb))
    tol = 1e-5 * (np.abs(act["c0b"]) @ np.abs(hw) + 1)
    assert np.all(np.abs(net_run["pred"].cpu().numpy() - ref) <= tol)


def test_unet_backward_matches_oracle(S, net_run):
    """Parameter gradients against the oracle's chain rule evaluated on the GPU's
    activations.  The GPU keeps every intermediate gradient in BF16 (2^-9
    relative per layer, through up to 20 layers), so tensors are compared by
    relative L2 error and cosine similarity rather than elementwise."""
    table, act = _layer_inputs(net_run)
    pred = net_run["pred"].cpu().numpy().astype(np.float64)
    target = net_run["target"].cpu().numpy().astype(np.float64)
    P = {k: (w_bf(w) if k != "head" else w.astype(np.float32).astype(np.float64), b)
         for k, (w, b) in net_run["params"].items()}
    ref = U.backward(P, act, pred, target, C0)
    got = S.unflatten_params(net_run["grads"], table, C0)
    assert float(net_run["loss"].item()) == pytest.approx(U.loss(pred, target), rel=1e-6)
    for name in [t[0] for t in table] + ["head"]:
        for which in (0, 1):
            r = np.asarray(ref[name][which], dtype=np.float64).ravel()
            g = np.asarray(got[name][which], dtype=np.float64).ravel()
            rel = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-30)
            cos = float(g @ r / max(np.linalg.norm(g) * np.linalg.norm(r), 1e-30))
            assert rel < 0.03 and cos > 0.999, (name, which, rel, cos)


def test_unet_backward_fluence_weighted_matches_oracle(S):
    """The fluence-weighted loss (SPNN_OPT_LOSS_FLUENCE_WEIGHT): loss value and
    parameter gradients against the oracle's weighted chain rule on the GPU's
    own activations, same bounds as the unweighted comparison."""
    rng = np.random.default_rng(12)
    params = U.init_params(C0, 23)
    net = S.UNet(C0, N, BATCH)
    net.set_params(S.flatten_params(params, C0))
    mask = (rng.random((BATCH, N, N, N)) < 0.7).astype(np.uint8)
    optics = np.stack([rng.uniform(0.1, 2.0, BATCH), rng.uniform(0.001, 0.05, BATCH),
                       rng.uniform(0.0, 0.9, BATCH)], axis=1).astype(np.float32)
    x = zeros_act(BATCH, N, N, N, 16)
    S.spnn_pack_input(torch.from_numpy(mask).cuda(), torch.from_numpy(optics).cuda(), x)
    pred = torch.zeros((BATCH, N, N, N), dtype=torch.float32, device="cuda")
    net.forward(x, pred)
    acts = [net.activation(i, BATCH) for i in range(20)]
    # log-fluence-like targets: a depth decay plus noise, so the weights span decades
    z = np.arange(N, dtype=np.float64)[None, :, None, None]
    tgt = -0.15 * z + rng.standard_normal((BATCH, N, N, N)) * 0.3
    target = torch.from_numpy(tgt.astype(np.float32)).cuda()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    try:
        S.spnn_set_option("loss_fluence_weight", 1)
        net.backward(target, loss)
        S.spnn_status()
    finally:
        S.spnn_set_option("loss_fluence_weight", 0)
    grads = net.get_grads()
    net.close()
    table = U.layer_table(C0)
    act = {"x": f64(x)}
    for (name, *_), a in zip(table, acts):
        act[name] = f64(a)
    p64 = pred.cpu().numpy().astype(np.float64)
    t64 = target.cpu().numpy().astype(np.float64)
    P = {k: (w_bf(w) if k != "head" else w.astype(np.float32).astype(np.float64), b) for k, (w, b) in params.items()}
    ref = U.backward(P, act, p64, t64, C0, fluence_weighted=True)
    got = S.unflatten_params(grads, table, C0)
    assert float(loss.item()) == pytest.approx(U.loss(p64, t64, fluence_weighted=True), rel=1e-5)
    assert float(loss.item()) != pytest.approx(U.loss(p64, t64), rel=1e-2)
    for name in [t[0] for t in table] + ["head"]:
        for which in (0, 1):
            r = np.asarray(ref[name][which], dtype=np.float64).ravel()
            g = np.asarray(got[name][which], dtype=np.float64).ravel()
            rel = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-30)
            cos = float(g @ r / max(np.linalg.norm(g) * np.linalg.norm(r), 1e-30))
            assert rel < 0.03 and cos > 0.999, (name, which, rel, cos)


def test_unet_adam_step(S, net_run):
    net = net_run["net"]
    p0 = net.get_params().astype(np.float64)
    g = net_run["grads"].astype(np.float64)
    net.adam(1e-3)
    S.spnn_status()
    p1 = net.get_params().astype(np.float64)
    ref, _, _ = U.adam_step(p0, g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
    np.testing.assert_allclose(p1, ref, rtol=1e-5, atol=1e-7)
    net.set_params(net_run["flat"])


def test_unet_training_reduces_loss(S):
    """Thirty Adam steps on one batch with a smooth target (a function of the
    mask and depth) must cut the loss well below its start."""
    rng = np.random.default_rng(12)
    net = S.UNet(C0, N, BATCH)
    net.set_params(S.flatten_params(U.init_params(C0, 4), C0))
    mask = (rng.random((BATCH, N, N, N)) < 0.7).astype(np.uint8)
    optics = np.tile(np.array([[0.5, 0.005, 0.7]], dtype=np.float32), (BATCH, 1))
    x = zeros_act(BATCH, N, N, N, 16)
    S.spnn_pack_input(torch.from_numpy(mask).cuda(), torch.from_numpy(optics).cuda(), x)
    z = (np.arange(N) + 0.5) / N
    tgt = -2.0 * z[None, :, None, None] + 0.3 * mask
    target = torch.from_numpy(tgt.astype(np.float32)).cuda()
    pred = torch.zeros((BATCH, N, N, N), dtype=torch.float32, device="cuda")
    losses = []
    for _ in range(30):
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        net.forward(x, pred)
        net.backward(target, loss)
        net.adam(2e-3)
        losses.append(float(loss.item()))
    S.spnn_status()
    net.close()
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.3 * losses[0], losses


@pytest.mark.parametrize("subtiles,planes", [(1, 2), (1, 4), (2, 2), (2, 4), (4, 2)])
def test_conv3_tilings_agree_with_oracle(S, subtiles, planes):
    """Every conv3 tiling (128-row subtiles per CTA, chunk planes per K-step)
    computes the same forward and input gradient within the bound."""
    rng = np.random.default_rng(13)
    B, D, H, W, c0, c1, co = 1, 4, 32, 32, 32, 32, 32
    x0, x1 = bf(rnd(rng, (B, D, H, W, c0))), bf(rnd(rng, (B, D, H, W, c1)))
    w = rnd(rng, (27, c0 + c1, co), 0.1)
    b = rnd(rng, co, 0.5)
    try:
        S.spnn_set_option("conv_subtiles", subtiles)
        S.spnn_set_option("conv_planes", planes)
        S.spnn_set_option("stage_kb", 200)
        y = zeros_act(B, D, H, W, co)
        S.spnn_layer_forward(S.CONV3, (B, D, H, W), x0, x1, packed(S, 0, c0 + c1, co, 0, w),
                             torch.tensor(b, dtype=torch.float32, device="cuda"), co, True, y)
        dx0, dx1 = zeros_act(B, D, H, W, c0), zeros_act(B, D, H, W, c1)
        S.spnn_layer_dgrad(S.CONV3, (B, D, H, W), y, packed(S, 0, c0 + c1, co, 1, w), c0, c1, dx0, dx1=dx1)
        S.spnn_status()
    finally:
        for k in ("conv_subtiles", "conv_planes", "stage_kb"):
            S.spnn_set_option(k, 0)
    xin = np.concatenate([f64(x0), f64(x1)], axis=-1)
    check(f64(y), U.relu(U.conv3(xin, w_bf(w), b)), U.conv3(np.abs(xin), np.abs(w_bf(w)), np.abs(b)), what="fwd")
    g = U.conv3_dgrad(f64(y), w_bf(w))
    ga = U.conv3_dgrad(np.abs(f64(y)), np.abs(w_bf(w)))
    check(np.concatenate([f64(dx0), f64(dx1)], axis=-1), g, ga, what="dgrad")


# (plane, dz, dy) row groups of 2 .. 10 planes per CTA, one or two sources, and
# plane splits across CTAs (co = 64: at most 3 planes per CTA, so 64 channels
# split 3 + 3 + 2, the last CTA's box running one zero plane past the source);
# halo 2 forces the halo kernel where the automatic choice takes the per-tap one,
# and 16 + 16 -> 32 runs 32-voxel x-runs (two CTAs per SM) over two sources
@pytest.mark.parametrize("c0,c1,co,halo", [(32, 0, 32, 1), (32, 32, 32, 1), (16, 0, 32, 1), (32, 32, 32, 0),
                                           (48, 0, 32, 1), (80, 0, 16, 1), (64, 0, 64, 2), (40, 24, 64, 2),
                                           (32, 0, 80, 2), (64, 64, 64, 2), (16, 16, 32, 1)])
def test_conv3_wgrad_halo_kernel(S, c0, c1, co, halo):
    """conv3 weight and bias gradients with halo K-steps (all 27 taps from one
    input box and three shifted output-gradient boxes per 16-voxel run) and
    with the per-tap kernel, against the oracle."""
    rng = np.random.default_rng(14)
    B, D, H, W = 2, 4, 8, 32
    x0 = bf(rnd(rng, (B, D, H, W, c0)))
    x1 = bf(rnd(rng, (B, D, H, W, c1))) if c1 else None
    dy = bf(rnd(rng, (B, D, H, W, co)))
    xin = f64(x0) if x1 is None else np.concatenate([f64(x0), f64(x1)], axis=-1)
    ref_w, ref_b = U.conv3_wgrad(xin, f64(dy))
    abs_w, abs_b = U.conv3_wgrad(np.abs(xin), np.abs(f64(dy)))
    dw = torch.zeros((27, c0 + c1, co), dtype=torch.float32, device="cuda")
    db = torch.zeros(co, dtype=torch.float32, device="cuda")
    try:
        S.spnn_set_option("wgrad_halo", halo)
        S.spnn_layer_wgrad(S.CONV3, (B, D, H, W), x0, x1, dy, dw, db)
        S.spnn_status()
    finally:
        S.spnn_set_option("wgrad_halo", 1)
    check(dw.cpu().numpy().astype(np.float64), ref_w, abs_w, out_bf16=False, what="dw")
    check(db.cpu().numpy().astype(np.float64), ref_b, abs_b, out_bf16=False, what="db")


def test_rows_gemm_persistent_grid_sizes_agree(S):
    """The persistent rows GEMM claims tiles dynamically; the result of every
    tile is independent of the CTA that computes it, so grids of one CTA per
    tile and of 1, 2 or 3 times the resident CTAs give identical bits (conv3
    forward with concatenated input and bias, and the down layer's scatter
    input gradient with 128-column N tiles)."""
    rng = np.random.default_rng(31)
    B, D, H, W, c0, c1, co = 2, 8, 16, 32, 16, 16, 32
    x0 = bf(rnd(rng, (B, D, H, W, c0)))
    x1 = bf(rnd(rng, (B, D, H, W, c1)))
    pk = packed(S, S.CONV3, c0 + c1, co, 0, rnd(rng, (27, c0 + c1, co), 0.1))
    bias = torch.tensor(rnd(rng, co, 0.5), dtype=torch.float32, device="cuda")
    dy = bf(rnd(rng, (B, D // 2, H // 2, W // 2, 64)))
    pkd = packed(S, S.DOWN, 32, 64, 1, rnd(rng, (8, 32, 64), 0.1))
    outs = []
    try:
        for grid in (0, 1, 2, 3):
            S.spnn_set_option("rows_persistent", grid)
            y = zeros_act(B, D, H, W, co)
            S.spnn_layer_forward(S.CONV3, (B, D, H, W), x0, x1, pk, bias, co, True, y)
            dx = zeros_act(B, D, H, W, 32)
            S.spnn_layer_dgrad(S.DOWN, (B, D, H, W), dy, pkd, 32, 0, dx)
            S.spnn_status()
            outs.append((y.clone(), dx.clone()))
    finally:
        S.spnn_set_option("rows_persistent", 2)
    for y, dx in outs[1:]:
        assert torch.equal(y, outs[0][0]) and torch.equal(dx, outs[0][1])
    assert float(outs[0][0].float().abs().sum()) > 0 and float(outs[0][1].float().abs().sum()) > 0


@pytest.mark.parametrize("B,D,H,W", [(1, 2, 4, 64), (1, 16, 4, 16), (3, 1, 8, 32)])
def test_conv3_wgrad_halo_walks(S, B, D, H, W):
    """The halo weight gradient's K walk (x-runs, z within slabs of up to 8
    planes, y, slabs, samples): slabs of 2, two slabs of 8, slabs of 1 over
    several samples, four x-runs per row."""
    rng = np.random.default_rng(B * 100 + D)
    c0, co = 32, 32
    x0 = bf(rnd(rng, (B, D, H, W, c0)))
    dy = bf(rnd(rng, (B, D, H, W, co)))
    ref_w, ref_b = U.conv3_wgrad(f64(x0), f64(dy))
    abs_w, abs_b = U.conv3_wgrad(np.abs(f64(x0)), np.abs(f64(dy)))
    dw = torch.zeros((27, c0, co), dtype=torch.float32, device="cuda")
    db = torch.zeros(co, dtype=torch.float32, device="cuda")
    S.spnn_layer_wgrad(S.CONV3, (B, D, H, W), x0, None, dy, dw, db)
    S.spnn_status()
    check(dw.cpu().numpy().astype(np.float64), ref_w, abs_w, out_bf16=False, what="dw")
    check(db.cpu().numpy().astype(np.float64), ref_b, abs_b, out_bf16=False, what="db")


@pytest.mark.parametrize("subtiles,planes", [(1, 2), (1, 4), (2, 2), (2, 4)])
def test_conv3_full_halo_tiling(S, subtiles, planes):
    """The full-halo conv3 tiling (8 x 16 tiles, one box per plane block for
    all 27 taps) against the oracle, forward and input gradient."""
    rng = np.random.default_rng(15)
    B, D, H, W, c0, c1, co = 1, 4, 32, 32, 32, 32, 32
    x0, x1 = bf(rnd(rng, (B, D, H, W, c0))), bf(rnd(rng, (B, D, H, W, c1)))
    w = rnd(rng, (27, c0 + c1, co), 0.1)
    b = rnd(rng, co, 0.5)
    try:
        S.spnn_set_option("conv_full_halo", 1)
        S.spnn_set_option("conv_subtiles", subtiles)
        S.spnn_set_option("conv_planes", planes)
        S.spnn_set_option("stage_kb", 200)
        y = zeros_act(B, D, H, W, co)
        S.spnn_layer_forward(S.CONV3, (B, D, H, W), x0, x1, packed(S, 0, c0 + c1, co, 0, w),
                             torch.tensor(b, dtype=torch.float32, device="cuda"), co, True, y)
        dx0, dx1 = zeros_act(B, D, H, W, c0), zeros_act(B, D, H, W, c1)
        S.spnn_layer_dgrad(S.CONV3, (B, D, H, W), y, packed(S, 0, c0 + c1, co, 1, w), c0, c1, dx0, dx1=dx1)
        S.spnn_status()
    finally:
        for k in ("conv_full_halo", "conv_subtiles", "conv_planes", "stage_kb"):
            S.spnn_set_option(k, 0)
    xin = np.concatenate([f64(x0), f64(x1)], axis=-1)
    check(f64(y), U.relu(U.conv3(xin, w_bf(w), b)), U.conv3(np.abs(xin), np.abs(w_bf(w)), np.abs(b)), what="fwd")
    g = U.conv3_dgrad(f64(y), w_bf(w))
    ga = U.conv3_dgrad(np.abs(f64(y)), np.abs(w_bf(w)))
    check(np.concatenate([f64(dx0), f64(dx1)], axis=-1), g, ga, what="dgrad")
