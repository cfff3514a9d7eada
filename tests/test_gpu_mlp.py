"""Learned troubled-cell indicator on the GPU against the FP64 oracle:
features and TVB labels, FP32 training gradients, BF16 tensor-core
inference, training progress, and the fused indicator in the step."""
import numpy as np
import pytest

import crkdg_inputs as inp
from oracle import mlp as omlp
from oracle import tableaux as OTB
from oracle.dg2d import cfl_dt_2d, crkdg_step
from oracle.limiter import neighbour_averages, tvb_limit
from tests.pairing import from_planes, make_pair_2d, rel_err, to_planes

pytestmark = pytest.mark.gpu
OUT = {s: ("outflow",) for s in "WESN"}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2307_06471_gb300 import build
    build.build()


def _oracle_params(P):
    """Pack oracle params (W: out x in) into the library's FP32 vector."""
    parts = []
    for W, b in zip(P["W"], P["b"]):
        parts += [W.reshape(-1), b.reshape(-1)]
    return np.concatenate(parts).astype(np.float32)


def _unpack(vec):
    sizes = [(64, 40), (64, 64), (64, 64), (1, 64)]
    P = {"W": [], "b": []}
    o = 0
    for (a, b) in sizes:
        P["W"].append(vec[o:o + a * b].astype(np.float64).reshape(a, b))
        o += a * b
        P["b"].append(vec[o:o + a].astype(np.float64))
        o += a
    return P


def _state(nx=45, ny=37, seed=41, amp=0.3):
    return inp.random_modal_state(ny, nx, 2, "P", "euler", seed=seed, amp=amp)


def test_features_and_labels_match_oracle():
    import torch
    nx, ny, M = 45, 37, 20.0
    gs, dg = make_pair_2d(nx, ny, (0, 1.5, 0, 1.0), 2, "P", "euler", "ssprk3", OUT, "f64")
    u = _state(nx, ny)
    gs.set_state(to_planes(u), 0.0)
    X = torch.zeros(nx * ny, 40, dtype=torch.float32, device="cuda")
    y = torch.zeros(nx * ny, dtype=torch.float32, device="cuda")
    gs.features(X.data_ptr(), y.data_ptr(), M)
    nb = neighbour_averages(dg, u[..., 0], 0.0)
    want = omlp.features(u, nb, M, max(dg.dx, dg.dy))
    got = X.cpu().numpy().astype(np.float64)
    # FP32 features of FP64 averages: differences round at ulp(avg) / s_q
    assert np.max(np.abs(got[:, :36] - want[:, :36])) < 1e-5
    assert np.max(np.abs(got[:, 36:] - want[:, 36:])) < 2e-5
    _, flags = tvb_limit(dg, u, M, 0.0)
    assert flags.any() and not flags.all()
    assert np.array_equal(y.cpu().numpy().reshape(ny, nx) > 0.5, flags)


def test_training_gradient_matches_oracle():
    import torch
    from paper_2307_06471_gb300 import binding as B
    rng = np.random.default_rng(5)
    P = omlp.init_params(rng)
    vec = _oracle_params(P)
    n = 300
    Xh = rng.normal(size=(n, 40)).astype(np.float32)
    yh = (rng.uniform(size=n) < 0.3).astype(np.float32)
    net = B.MLP(seed=1)
    net.set_params(vec)
    X = torch.tensor(Xh, device="cuda")
    y = torch.tensor(yh, device="cuda")
    loss, g = net.loss_grad(X.data_ptr(), y.data_ptr(), n, pos_weight=2.5)
    P32 = _unpack(vec)
    z, cache = omlp.forward(P32, Xh.astype(np.float64))
    L, dz = omlp.bce_with_logits(z, yh.astype(np.float64), pos_weight=2.5)
    G = omlp.backward(P32, cache, dz)
    want = _oracle_params(G).astype(np.float64)
    assert loss == pytest.approx(L, rel=1e-5)
    assert np.linalg.norm(g - want) / np.linalg.norm(want) < 1e-5
    net.close()


def test_bf16_inference_matches_oracle_forward():
    import torch
    from paper_2307_06471_gb300 import binding as B
    rng = np.random.default_rng(6)
    P = omlp.init_params(rng)
    vec = _oracle_params(P)
    n = 1000
    Xh = rng.normal(size=(n, 40)).astype(np.float32)
    net = B.MLP(seed=1)
    net.set_params(vec)
    X = torch.tensor(Xh, device="cuda")
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    net.predict(X.data_ptr(), n, out.data_ptr())
    z, _ = omlp.forward(_unpack(vec), Xh.astype(np.float64))
    zg = out.cpu().numpy()
    scale = max(1.0, np.max(np.abs(z)))
    # BF16 weights and activations, FP32 accumulation
    assert np.max(np.abs(zg - z)) < 0.05 * scale
    assert np.mean(np.abs(zg - z)) < 0.01 * scale
    net.close()


def test_tcgen05_inference_matches_mma_sync_and_oracle():
    """The fifth-generation tensor-core inference (tiles of 512 samples,
    tcgen05 products into tensor memory) against the mma.sync inference on
    the same BF16 network (same BF16 roundings of weights and activations;
    only the FP32 accumulation order differs) and against the FP64 oracle
    forward with the BF16 bands of the test above; 1000 samples (a partial
    last tile) and one sample."""
    import torch
    from paper_2307_06471_gb300 import binding as B
    rng = np.random.default_rng(16)
    P = omlp.init_params(rng)
    vec = _oracle_params(P)
    net = B.MLP(seed=1)
    net.set_params(vec)
    for n in (1000, 1):
        Xh = rng.normal(size=(n, 40)).astype(np.float32)
        X = torch.tensor(Xh, device="cuda")
        a = torch.zeros(n, dtype=torch.float32, device="cuda")
        b = torch.full((n,), -7.0, dtype=torch.float32, device="cuda")
        net.predict(X.data_ptr(), n, a.data_ptr())
        net.predict_tc(X.data_ptr(), n, b.data_ptr())
        za, zb = a.cpu().numpy(), b.cpu().numpy()
        z, _ = omlp.forward(_unpack(vec), Xh.astype(np.float64))
        scale = max(1.0, np.max(np.abs(z)))
        assert np.all(np.isfinite(zb))
        assert np.max(np.abs(zb - za)) < 0.02 * scale
        assert np.max(np.abs(zb - z)) < 0.05 * scale
        assert np.mean(np.abs(zb - z)) < 0.01 * scale
    net.close()


def test_training_learns_a_separable_rule():
    import torch
    from paper_2307_06471_gb300 import binding as B
    rng = np.random.default_rng(7)
    n = 8192
    Xh = rng.normal(size=(n, 40)).astype(np.float32)
    yh = ((Xh[:, 0] + 0.5 * Xh[:, 5] - Xh[:, 37]) > 0.3).astype(np.float32)
    X = torch.tensor(Xh, device="cuda")
    y = torch.tensor(yh, device="cuda")
    net = B.MLP(seed=3)
    l0, _ = net.loss_grad(X.data_ptr(), y.data_ptr(), n)
    l1 = net.train(X.data_ptr(), y.data_ptr(), n, epochs=8, batch=256, lr=2e-3, seed=11)
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    net.predict(X.data_ptr(), n, out.data_ptr())
    acc = np.mean((out.cpu().numpy() > 0) == (yh > 0.5))
    assert l1 < 0.3 * l0 and acc > 0.95
    net.close()


@pytest.mark.parametrize("where", ["fused", "pass_tcgen05", "pass_mma_sync"])
@pytest.mark.parametrize("mode", ["always", "never", "tvb_band"])
def test_fused_indicator_decisions(mode, where):
    """A network whose output is a constant logit forces the decision (all
    cells limited / none); a band covering every logit leaves it to TVB.  The
    indicator runs fused into the step's load (mma.sync) or in the limiter
    pass (tcgen05 or mma.sync); nx = 300 leaves a partial tile."""
    import torch
    from paper_2307_06471_gb300 import binding as B
    nx, ny, M = 300, 40, 20.0
    gs, dg = make_pair_2d(nx, ny, (0, 1.0, 0, 1.0), 2, "P", "euler", "ssprk3", OUT, "f32")
    gs.set_limit_mode(B.LIMIT_FUSED if where == "fused" else B.LIMIT_PASS)
    gs.set_indicator_engine(B.MLP_MMA_SYNC if where == "pass_mma_sync" else B.MLP_TCGEN05)
    u = _state(nx, ny, seed=42)
    u = from_planes(to_planes(u).astype(np.float32).astype(np.float64))
    vec = np.zeros(11009, dtype=np.float32)
    vec[-1] = {"always": 10.0, "never": -10.0, "tvb_band": 0.0}[mode]
    net = B.MLP()
    net.set_params(vec)
    gs.set_state(to_planes(u), 0.0)
    gs.limit(M)
    if mode == "tvb_band":
        gs.set_indicator(net, -1e30, 1e30)
    else:
        gs.set_indicator(net, -1.0, 1.0)
    dt = 0.2 * cfl_dt_2d(dg, u, 1.0)
    gs.step(dt)
    # get_state applies the pending end-of-step limit with the TVB test
    got = from_planes(gs.get_state())
    if mode == "tvb_band":
        lim = tvb_limit(dg, u, M, 0.0)[0]
    else:
        force = np.full((ny, nx), mode == "always")
        lim = tvb_limit(dg, u, M, 0.0, force=force)[0]
    want = tvb_limit(dg, crkdg_step(dg, lim, 0.0, dt, OTB.SSPRK3), M, dt)[0]
    assert rel_err(got, want) < 2e-5
    assert gs.sync() == (0, 0)    # no bounded wait ran out
    net.close()


@pytest.mark.parametrize("engine,nx", [("tcgen05", 300), ("tcgen05", 298), ("mma_sync", 300)])
def test_pass_decisions_follow_the_network_logits(engine, nx):
    """A seeded untrained network whose logits spread over both signs, with
    the band [z_lo, z_hi] between the 30 % and 70 % quantiles of the logits:
    the limiter pass (tcgen05 or mma.sync inference) limits a cell when its
    logit, from the same features by the separate mma.sync inference, is
    above z_hi, keeps it when below z_lo, and leaves the TVB test to decide
    in between.  A cell may differ from that only where its logit lies
    within 2 % of the logit scale of a band edge (BF16 rounding and the
    accumulation order).  nx = 300 and 298: a partial last tile of 512 and
    of 32 cells, rows of 16-byte multiples and not."""
    import torch
    from paper_2307_06471_gb300 import binding as B
    ny, M = 40, 20.0
    gs, dg = make_pair_2d(nx, ny, (0, 1.0, 0, 1.0), 2, "P", "euler", "ssprk3", OUT, "f32")
    gs.set_indicator_engine(B.MLP_TCGEN05 if engine == "tcgen05" else B.MLP_MMA_SYNC)
    u = _state(nx, ny, seed=43)
    u = from_planes(to_planes(u).astype(np.float32).astype(np.float64))
    gs.set_state(to_planes(u), 0.0)
    n = nx * ny
    X = torch.zeros(n, 40, dtype=torch.float32, device="cuda")
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    gs.features(X.data_ptr(), y.data_ptr(), M)
    net = B.MLP(seed=5)
    zt = torch.zeros(n, dtype=torch.float32, device="cuda")
    net.predict(X.data_ptr(), n, zt.data_ptr())
    z = zt.cpu().numpy().astype(np.float64).reshape(ny, nx)
    z_lo, z_hi = np.quantile(z, 0.3), np.quantile(z, 0.7)
    assert z_lo < z_hi
    gs.set_indicator(net, z_lo, z_hi)
    gs.limit(M)
    gs.apply_limit()
    got = from_planes(gs.get_state())
    assert gs.sync() == (0, 0)
    tvb_flags = tvb_limit(dg, u, M, 0.0)[1]
    decide = np.where(z > z_hi, True, np.where(z < z_lo, False, tvb_flags))
    want = tvb_limit(dg, u, M, 0.0, force=decide)[0]
    # the decisions matter: forcing changes the outcome against plain TVB
    assert np.count_nonzero(decide != tvb_flags) > 0.05 * n
    scale = np.max(np.abs(want), axis=(0, 1, 3))
    bad = np.any(np.abs(got - want) > 2e-5 * scale[None, None, :, None], axis=(2, 3))
    zs = max(1.0, float(np.max(np.abs(z))))
    near = (np.abs(z - z_hi) < 0.02 * zs) | (np.abs(z - z_lo) < 0.02 * zs)
    assert not np.any(bad & ~near), np.argwhere(bad & ~near)[:5]
    assert np.count_nonzero(bad) <= 0.01 * n
    net.close()
