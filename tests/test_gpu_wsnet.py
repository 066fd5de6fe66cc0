"""GPU checks of the warm-start network against the FP64 numpy oracle.

Single convolutions (lbm_conv3d_bf16: forward, data gradient, weight
gradient) on the tensor cores, for channel pairs covering every operand
shape and swizzle mode, on a ragged multi-tile volume.  Inputs and weights are
rounded to BF16 on the host and the oracle gets the same rounded values, so
the only differences are in the arithmetic: the products of two BF16 values
are exact in FP32; each FP32 addition rounds by at most 2^-24 of the running
sum, whose magnitude is at most S = the same sum over absolute values; the
forward and data-gradient outputs are then rounded to BF16 (2^-8 relative,
half an ulp of 8 significant bits, times two for the rounding of the sum
before it).  Allowing 2^8 rounding steps on the path of one sum gives
|got - ref| <= 2^-8 |ref| + 2^-16 S.

The whole network (4 levels, 32 base channels): loss and every parameter
gradient against the FP64 oracle.  Here BF16 rounds every activation and
gradient tensor (relative 2^-9) on a path of about 30 layers forward and
back, and a rounding can move a ReLU input across zero; the test states the
per-layer relative L2 error of the gradient at <= 0.06 and the loss at 1e-2."""
import numpy as np
import pytest

from oracle import wsnet_oracle as N

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    t.cuda.set_device(0)
    import __graft_entry__

    __graft_entry__.build()
    return t


def _bf16(torch, a):
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16)


def _padded(torch, x):
    """[B][C][Z][Y][X] float -> device BF16 [B][Z+2][Y+2][X+2][C] with a zero border,
    and the BF16-rounded values as float64 (same shape as x)."""
    B, C, Z, Y, X = x.shape
    t = torch.zeros((B, Z + 2, Y + 2, X + 2, C), dtype=torch.bfloat16, device="cuda")
    xb = _bf16(torch, x)
    t[:, 1:-1, 1:-1, 1:-1, :] = xb.permute(0, 2, 3, 4, 1).cuda()
    return t, xb.double().numpy()


def _unpad(t):
    return t[:, 1:-1, 1:-1, 1:-1, :].permute(0, 4, 1, 2, 3).double().cpu().numpy()


PAIRS = [(32, 32), (32, 64), (64, 32), (64, 128), (128, 256), (256, 128), (256, 256), (32, 256)]
SHAPE = (2, 6, 7, 9)  # B, Z, Y, X: 2 * 8 * 9 * 11 padded rows = 13 tiles of 128 with a ragged tail


@pytest.mark.parametrize("cin,cout", PAIRS)
def test_conv_layer_matches_oracle(torch, cin, cout):
    from paper_1806_10589_gb300 import conv3d_bf16

    B, Z, Y, X = SHAPE
    rng = np.random.default_rng(cin * 7 + cout)
    a = rng.standard_normal((B, cin, Z, Y, X))
    g = rng.standard_normal((B, cout, Z, Y, X))
    w = rng.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin)
    bias = rng.standard_normal(cout).astype(np.float32)
    ta, a_r = _padded(torch, a)
    tg, g_r = _padded(torch, g)
    wb = _bf16(torch, w)
    w_r = wb.double().numpy().transpose(0, 2, 1)          # oracle layout W[co][ci][27]
    tw = wb.cuda().contiguous()
    tb = torch.tensor(bias).cuda()
    st = torch.cuda.current_stream()

    # forward with ReLU
    out = torch.full((B, Z + 2, Y + 2, X + 2, cout), 7.0, dtype=torch.bfloat16, device="cuda")
    conv3d_bf16(0, ta.data_ptr(), 0, tw.data_ptr(), tb.data_ptr(), 1, out.data_ptr(), B, X, Y, Z, cin, cout, st)
    got = _unpad(out)
    border = out.clone()
    border[:, 1:-1, 1:-1, 1:-1, :] = 0
    assert not border.any(), "border rows must be written 0"
    for b in range(B):
        ref = N.relu(N.conv(a_r[b], w_r, bias.astype(np.float64)))
        S = N.conv(np.abs(a_r[b]), np.abs(w_r), np.abs(bias.astype(np.float64)))
        err = np.abs(got[b] - ref) - (2.0 ** -8 * np.abs(ref) + 2.0 ** -16 * S)
        assert err.max() <= 0, ("forward", b, float(err.max()), float(np.abs(ref).max()))

    # data gradient
    gin = torch.full((B, Z + 2, Y + 2, X + 2, cin), 7.0, dtype=torch.bfloat16, device="cuda")
    conv3d_bf16(1, tg.data_ptr(), 0, tw.data_ptr(), 0, 0, gin.data_ptr(), B, X, Y, Z, cin, cout, st)
    got = _unpad(gin)
    for b in range(B):
        ref, _, _ = N.conv_backward(a_r[b], w_r, g_r[b])
        S, _, _ = N.conv_backward(np.abs(a_r[b]), np.abs(w_r), np.abs(g_r[b]))
        err = np.abs(got[b] - ref) - (2.0 ** -8 * np.abs(ref) + 2.0 ** -16 * S)
        assert err.max() <= 0, ("data gradient", b, float(err.max()), float(np.abs(ref).max()))

    # weight gradient (accumulated onto a preset value)
    gw = torch.full((cout, 27, cin), 0.5, dtype=torch.float32, device="cuda")
    conv3d_bf16(2, ta.data_ptr(), tg.data_ptr(), tw.data_ptr(), 0, 0, gw.data_ptr(), B, X, Y, Z, cin, cout, st)
    got = gw.double().cpu().numpy().transpose(0, 2, 1) - 0.5
    ref = np.zeros((cout, cin, 27))
    S = np.zeros((cout, cin, 27))
    for b in range(B):
        ref += N.conv_backward(a_r[b], w_r, g_r[b])[1]
        S += N.conv_backward(np.abs(a_r[b]), np.abs(w_r), np.abs(g_r[b]))[1]
    err = np.abs(got - ref) - (2.0 ** -16 * S + 2.0 ** -22)
    assert err.max() <= 0, ("weight gradient", float(err.max()), float(np.abs(ref).max()))


def test_conv_rejects_bad_shapes(torch):
    from paper_1806_10589_gb300 import LBMError, conv3d_bf16

    with pytest.raises(LBMError):
        conv3d_bf16(0, 1, 0, 1, 0, 0, 1, 1, 4, 4, 4, 48, 32)
    with pytest.raises(LBMError):
        conv3d_bf16(2, 1, 0, 1, 0, 0, 1, 1, 4, 4, 4, 32, 32)  # weight gradient needs the output gradient


@pytest.fixture(scope="module")
def net(torch):
    from paper_1806_10589_gb300 import WarmStartNet

    n = WarmStartNet(4, 32, stream=torch.cuda.current_stream())
    yield n
    n.close()


def _he(n_levels, base, seed):
    rng = np.random.default_rng(seed)
    parts = []
    for co, ci in N.layer_shapes(n_levels, base):
        parts.append(rng.standard_normal(co * 27 * ci) * np.sqrt(2.0 / (27 * ci)))
        parts.append(0.05 * rng.standard_normal(co))
    return np.concatenate(parts).astype(np.float32)


def test_param_count(net):
    assert net.n_params == N.n_params(4, 32)
    assert net.layer_shapes() == N.layer_shapes(4, 32)


def test_forward_matches_oracle(net):
    rng = np.random.default_rng(1)
    mask = (rng.random((16, 8, 8)) < 0.35).astype(np.uint8)
    p = _he(4, 32, 11)
    net.set_params(p)
    y = net.predict(mask)
    ref = N.forward(p.astype(np.float64), 1.0 - mask, 4, 32)
    assert np.all(y[:, mask == 1] == 0)
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert rel <= 0.03, rel


def test_loss_and_gradient_match_oracle(net):
    rng = np.random.default_rng(2)
    B, shape = 2, (16, 8, 8)
    masks = (rng.random((B,) + shape) < 0.35).astype(np.uint8)
    targets = rng.standard_normal((B, N.NOUT) + shape).astype(np.float32)
    targets[:, 3][rng.random((B,) + shape) < 0.3] = np.nan  # entries without a target
    p = _he(4, 32, 12)
    net.set_params(p)
    loss, g = net.loss_grad(masks, targets)
    # one normalisation by the batch's total pore count
    npore = float((masks == 0).sum())
    ref_loss, ref_g = 0.0, np.zeros(p.size)
    for b in range(B):
        nb = float((masks[b] == 0).sum())
        lb, gb = N.loss_and_grad(p.astype(np.float64), 1.0 - masks[b], targets[b], 4, 32)
        ref_loss += lb * nb / npore
        ref_g += gb * nb / npore
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss, (loss, ref_loss)
    k = 0
    for li, (co, ci) in enumerate(N.layer_shapes(4, 32)):
        n = co * 27 * ci + co
        a, r = g[k:k + n], ref_g[k:k + n]
        rel = np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-30)
        assert rel <= 0.06, (li, co, ci, rel)
        k += n


def test_training_reduces_loss(net):
    rng = np.random.default_rng(5)
    masks = (rng.random((6, 8, 8, 8)) < 0.3).astype(np.uint8)
    pore = 1.0 - masks.astype(np.float32)
    t = np.stack([pore * 0.5, pore * -0.2, pore * (1.0 + 0.1 * np.arange(8)[None, :, None, None]), pore * 2.0],
                 axis=1)
    net.set_params(_he(4, 32, 3) * 0.5)
    hist = net.train(masks, t.astype(np.float32), epochs=60, batch=3, lr=1e-3, seed=1)
    assert np.isfinite(hist).all()
    assert hist[-1] < 0.2 * hist[0], hist[[0, -1]]


def test_training_is_deterministic(net):
    """The weight and bias gradients are summed per row split and the splits
    added in a fixed order (no floating-point atomics), so the same data, start
    and sample order give bitwise the same gradients and the same trained
    parameters."""
    rng = np.random.default_rng(9)
    masks = (rng.random((4, 16, 16, 16)) < 0.3).astype(np.uint8)
    pore = 1.0 - masks.astype(np.float32)
    t = np.stack([pore * 0.3, pore * rng.standard_normal(masks.shape).astype(np.float32) * 0.1, pore * -0.2,
                  pore * 1.5], axis=1).astype(np.float32)
    p0 = _he(4, 32, 11) * 0.5
    runs = []
    for _ in range(2):
        net.set_params(p0)
        _, g = net.loss_grad(masks, t)
        hist = net.train(masks, t, epochs=3, batch=2, lr=1e-3, seed=3)
        runs.append((g, hist, net.params()))
    (g0, h0, q0), (g1, h1, q1) = runs
    assert np.abs(g0).max() > 0
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(q0, q1)
    assert not np.array_equal(q0, p0)


def test_interior_crops_of_the_training_data(torch):
    """With a margin the inputs and targets are the interior crops of the
    steady states: the crop's velocity is the whole box's (over u_D of the
    whole box), and its plane drops add up to the pressure difference between
    the crop's first and last planes."""
    from lbm_inputs import sphere_pack
    from paper_1806_10589_gb300 import Batch, Lattice, warmstart as ws

    st = torch.cuda.current_stream()
    m = sphere_pack(24, 3.0, 5.0, 0.4, seed=41, cache=False)[0]
    inputs, targets, ks = ws.steady_targets(Batch, [m], 0.8, 1e-4, 600, stream=st, margin=4)
    assert inputs[0].shape == (16, 16, 16)
    np.testing.assert_array_equal(inputs[0], m[4:-4, 4:-4, 4:-4])
    Q = 1e-4 * int((m[0] == 0).sum())
    uD = Q / 24 ** 2
    with Lattice(m, 0.8, "mrt", "fp32", stream=st) as lat:
        lat.set_flux_bc(Q)
        lat.step(600)
        rho, ux, uy, uz = lat.fields()
    c = (slice(4, -4),) * 3
    np.testing.assert_allclose(targets[0, 2], (uz[c] / uD).astype(np.float32), rtol=1e-5, atol=1e-6)
    prof = ws.pressure_profile(targets[0, 3], inputs[0], uD * 16 * 16, 0.8, rho_out=0.0)
    pbar = ws.plane_means(rho[c], inputs[0])
    np.testing.assert_allclose(prof[0] - prof[-1], pbar[0] - pbar[-1], rtol=1e-4)


def test_warm_start_pipeline_small(net, torch):
    """End to end at small scale: steady targets from the batched LBM, a short
    training run, Kozeny-Carman calibration and a warm-started lattice that
    reaches the 0.1 % rule of a reference run."""
    from lbm_inputs import sphere_pack
    from paper_1806_10589_gb300 import Batch, Lattice, convergence as cv, warmstart as ws

    st = torch.cuda.current_stream()
    masks = [sphere_pack(32, 5.0, 8.0, 0.4, seed=300 + k, cache=False)[0] for k in range(8)]
    inputs, targets, ks = ws.steady_targets(Batch, masks, 0.8, 1e-4, 3000, stream=st)
    assert all(a.shape == m.shape for a, m in zip(inputs, masks))
    assert np.isfinite(targets[:, :3]).all() and (ks > 0).all()
    # G is defined (finite) on the pore voxels of every plane but the last, and
    # its plane drops add up to the steady pressure drop: the permeability they
    # imply is the one the LBM reports
    m = np.stack(masks)
    defined = np.zeros(m.shape, bool)
    defined[:, :-1] = m[:, :-1] == 0
    np.testing.assert_array_equal(np.isfinite(targets[:, 3]), defined)
    for k in range(len(masks)):
        Q = 1e-4 * int((masks[k][0] == 0).sum())
        prof = ws.pressure_profile(targets[k, 3], masks[k], Q, 0.8)
        k_t = cv.permeability(Q, masks[k].shape, 0.8, prof[0], prof[-1])
        assert abs(k_t - ks[k]) <= 1e-4 * ks[k], (k, k_t, ks[k])
    c_kc = ws.fit_kc(masks, ks)
    assert c_kc > 0
    net.set_params(ws.he_init(net, 0))
    hist = net.train(np.stack(inputs), targets, epochs=20, batch=4, lr=1e-3, seed=0)
    assert hist[-1] < hist[0]
    m = sphere_pack(32, 5.0, 8.0, 0.4, seed=999, cache=False)[0]
    Q = 1e-4 * int((m[0] == 0).sum())
    with Lattice(m, 0.8, "mrt", "fp32", stream=st) as lat:
        lat.set_flux_bc(Q)
        ref = cv.run_to_residual(lat, Q, 0.8, lag=500, tol=1e-6, max_steps=40000)
    res = ws.warm_vs_cold(Lattice, net, m, Q, 0.8, c_kc, ref["k"], stream=st, max_steps=40000)
    info = {"res": res, "k_ref": ref["k"]}
    assert res["cold"]["reached"] and res["warm"]["reached"], info
    assert abs(res["warm"]["k"] - ref["k"]) <= 1e-3 * ref["k"]


def test_adam_steps_match_the_published_update(torch):
    """Two training steps (one batch holding every sample, so each epoch is
    one step) against Adam as Kingma and Ba define it, fed with the gradients
    the library reports at the same parameters: m = b1 m + (1 - b1) g,
    v = b2 v + (1 - b2) g^2, p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
    The weight gradients are FP32 atomic sums whose order varies between
    calls, so only parameters whose gradient is well above that noise
    (|g| > 1e-3 of the layer's max|g| in both steps) are compared, at 2e-3 of
    the step size."""
    from paper_1806_10589_gb300 import WarmStartNet

    rng = np.random.default_rng(8)
    masks = (rng.random((2, 8, 8, 8)) < 0.3).astype(np.uint8)
    t = rng.standard_normal((2, N.NOUT, 8, 8, 8)).astype(np.float32)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    with_net = WarmStartNet(2, 32, stream=torch.cuda.current_stream())
    try:
        p0 = _he(2, 32, 21)
        with_net.set_params(p0)
        _, g0 = with_net.loss_grad(masks, t)
        with_net.train(masks, t, epochs=1, batch=2, lr=lr, seed=0)
        p1 = with_net.params()
        _, g1 = with_net.loss_grad(masks, t)
        # a second epoch continues the same Adam state
        with_net.train(masks, t, epochs=1, batch=2, lr=lr, seed=0)
        p2 = with_net.params()
    finally:
        with_net.close()
    g0, g1 = g0.astype(np.float64), g1.astype(np.float64)
    m1, v1 = (1 - b1) * g0, (1 - b2) * g0 ** 2
    want1 = p0 - lr * (m1 / (1 - b1)) / (np.sqrt(v1 / (1 - b2)) + eps)
    m2, v2 = b1 * m1 + (1 - b1) * g1, b2 * v1 + (1 - b2) * g1 ** 2
    want2 = p1 - lr * (m2 / (1 - b1 ** 2)) / (np.sqrt(v2 / (1 - b2 ** 2)) + eps)
    # "well above the noise": per layer (gradient scales differ by orders of magnitude between layers)
    big = np.zeros(g0.size, bool)
    k = 0
    for co, ci in N.layer_shapes(2, 32):
        sl = slice(k, k + co * 27 * ci + co)
        big[sl] = (np.abs(g0[sl]) > 1e-3 * np.abs(g0[sl]).max()) & (np.abs(g1[sl]) > 1e-3 * np.abs(g1[sl]).max())
        k = sl.stop
    assert big.sum() > 0.5 * big.size
    assert np.abs(p1 - want1)[big].max() <= 2e-3 * lr
    assert np.abs(p2 - want2)[big].max() <= 2e-3 * lr
    # the first step moves every parameter by lr |g| / (|g| + eps) <= lr
    assert np.abs(p1 - p0).max() <= lr * (1 + 1e-3)


def test_exact_pressure_start_beats_cold(torch):
    """What the network's pressure output buys when it is exact: a stand-in
    network that returns the pack's own steady plane drops (and no velocity)
    starts the run at the right pressure, and the run meets the 0.1 % rule in
    well under half the steps of a cold start.  The trained network's gain is
    measured by the benchmark's warm-start leg."""
    from lbm_inputs import sphere_pack
    from paper_1806_10589_gb300 import Lattice, convergence as cv, warmstart as ws

    st = torch.cuda.current_stream()
    # long in z, so that the pressure (the slow mode, time ~ length^2) sets the pace
    m = sphere_pack((32, 32, 128), 5.0, 8.0, 0.4, seed=999, cache=False)[0]
    assert m.shape == (128, 32, 32)
    Q, tau = 1e-4 * int((m[0] == 0).sum()), 0.8
    with Lattice(m, tau, "mrt", "fp32", stream=st) as lat:
        lat.set_flux_bc(Q)
        ref = cv.run_to_residual(lat, Q, tau, lag=1000, tol=1e-6, max_steps=100000)
        rho, _, _, _ = lat.fields()
    G = np.nan_to_num(ws.drop_target(rho, m, Q, tau)).astype(np.float32)

    class Exact:
        def predict(self, mask):
            y = np.zeros((4,) + mask.shape, np.float32)
            y[3] = G
            return y

    cold = ws.run_start(Lattice, None, m, Q, tau, 1.0, ref["k"], "cold", stream=st, max_steps=100000)
    warm = ws.run_start(Lattice, Exact(), m, Q, tau, 1.0, ref["k"], "net_pressure", stream=st, max_steps=100000)
    assert cold["reached"] and warm["reached"], (cold, warm)
    assert warm["steps"] <= 0.5 * cold["steps"], (warm["steps"], cold["steps"])
    assert abs(warm["k"] - ref["k"]) <= 1e-3 * ref["k"]
