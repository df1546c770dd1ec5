"""GPU surrogate (BF16 tensor-core GEMMs, FP32 accumulation) against the
FP64 numpy reference of the same network.

Tolerances come from BF16 operand rounding (8-bit mantissa, ~2e-3 relative
per operand): forward relative L2 <= 1e-2 of the learned correction; per-tensor gradient relative L2 <= 5e-2; the
fixed rotation layer is an FP32 FFT per row (nine radix-2 stages each way,
~1e-6 relative rounding) and must match the FP64 DFT to <= 1e-5.
"""
import numpy as np
import pytest

import oracle.surrogate_ref as S
import sft_inputs as I
from paper_2501_06377_gb300 import build as B

pytestmark = pytest.mark.gpu

CFG = dict(channels=32, modes=16, blocks=2)


@pytest.fixture(scope="module")
def torch_mod():
    B.build()
    import torch
    assert torch.cuda.is_available()
    return torch


def _inputs(n, seed=1):
    x = np.stack([I.initial_map(S.H, S.W, seed=seed + i) for i in range(n)])
    draws = I.draw_realization_params(n, seed=seed)
    rng = np.random.default_rng(seed)
    p = np.array([[13.38 * rng.uniform(0.9, 1.1), -2.30 * rng.uniform(0.9, 1.1), -1.62 * rng.uniform(0.9, 1.1),
                   rng.uniform(10, 20), d[6]] for d in draws])
    y = x + rng.normal(0, 3.0, x.shape)
    return x, p, y


def _net(torch_mod, P):
    from paper_2501_06377_gb300.surrogate import Surrogate, flat_from_reference
    net = Surrogate(max_batch=4, **CFG)
    net.set_params(flat_from_reference(P, CFG["blocks"]))
    return net


def _cuda(torch_mod, a):
    return torch_mod.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_rotation_layer_is_fp32_accurate(torch_mod):
    P = S.init_params(C=CFG["channels"], M=CFG["modes"], L=CFG["blocks"], seed=0)
    P["Wd"][:] = 0.0
    P["bd"][:] = 0.0
    net = _net(torch_mod, P)
    x, p, _ = _inputs(2)
    out = torch_mod.empty((2, S.H, S.W), device="cuda")
    net.forward(_cuda(torch_mod, x), _cuda(torch_mod, p), out)
    ref = S.rotate(x.astype(np.float32).astype(np.float64), S.rotation_angles(p.astype(np.float32).astype(np.float64)))
    got = out.cpu().numpy()
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 1e-5, rel


def test_forward_matches_reference(torch_mod):
    P = S.init_params(C=CFG["channels"], M=CFG["modes"], L=CFG["blocks"], seed=2)
    P["Wd"] *= 50.0   # make the learned correction visible
    net = _net(torch_mod, P)
    x, p, _ = _inputs(2, seed=3)
    out = torch_mod.empty((2, S.H, S.W), device="cuda")
    net.forward(_cuda(torch_mod, x), _cuda(torch_mod, p), out)
    xr = x.astype(np.float32).astype(np.float64)
    pr = p.astype(np.float32).astype(np.float64)
    ref = S.forward(P, xr, pr, L=CFG["blocks"], M=CFG["modes"])
    r = S.rotate(xr, S.rotation_angles(pr))
    got = out.cpu().numpy()
    # the rotated map r is FP32-accurate (test above); the learned correction
    # x_next - r carries the BF16 rounding
    corr_err = np.linalg.norm((got - r) - (ref - r)) / np.linalg.norm(ref - r)
    assert corr_err <= 1e-2, corr_err


def test_gradients_match_reference(torch_mod):
    from paper_2501_06377_gb300.surrogate import unflatten_like
    P = S.init_params(C=CFG["channels"], M=CFG["modes"], L=CFG["blocks"], seed=4)
    P["Wd"] *= 50.0
    net = _net(torch_mod, P)
    x, p, y = _inputs(2, seed=5)
    loss, g = net.loss_grad(_cuda(torch_mod, x), _cuda(torch_mod, p), _cuda(torch_mod, y))
    xr, pr, yr = (a.astype(np.float32).astype(np.float64) for a in (x, p, y))
    rloss, rg = S.loss_and_grad(P, xr, pr, yr, L=CFG["blocks"], M=CFG["modes"])
    assert loss == pytest.approx(rloss, rel=2e-3)
    gg = unflatten_like(g, P, CFG["blocks"])
    for k in rg:
        if np.linalg.norm(rg[k]) == 0:
            assert np.linalg.norm(gg[k]) == 0, k
            continue
        rel = np.linalg.norm(gg[k] - rg[k]) / np.linalg.norm(rg[k])
        assert rel <= 5e-2, (k, rel)


def test_adamw_step_matches_reference(torch_mod):
    P = S.init_params(C=CFG["channels"], M=CFG["modes"], L=CFG["blocks"], seed=6)
    net = _net(torch_mod, P)
    from paper_2501_06377_gb300.surrogate import flat_from_reference
    x, p, y = _inputs(2, seed=7)
    xc, pc, yc = (_cuda(torch_mod, a) for a in (x, p, y))
    _, g = net.loss_grad(xc, pc, yc)
    before = net.get_params()
    net.train_step(xc, pc, yc, lr=1e-3, wd=1e-2)
    after = net.get_params()
    m = np.zeros_like(before, dtype=np.float64)
    v = np.zeros_like(m)
    Pf = {"a": before.astype(np.float64)}
    Pf, _, _ = S.adamw_step(Pf, {"a": g.astype(np.float64)}, {"a": m}, {"a": v}, 1, 1e-3, wd=1e-2)
    np.testing.assert_allclose(after, Pf["a"], rtol=0, atol=2e-6)
    del flat_from_reference


def test_training_reduces_loss(torch_mod):
    from paper_2501_06377_gb300.surrogate import Surrogate
    net = Surrogate(max_batch=4, seed=9, **CFG)
    x, p, y = _inputs(4, seed=11)
    xc, pc, yc = (_cuda(torch_mod, a) for a in (x, p, y))
    first = net.train_step(xc, pc, yc, lr=2e-3, want_loss=True)
    for _ in range(40):
        last = net.train_step(xc, pc, yc, lr=2e-3, want_loss=True)
    assert last < 0.5 * first, (first, last)


PROD = dict(channels=64, modes=48, blocks=4)   # the configuration of the fused inference kernel


def test_fused_forward_matches_reference(torch_mod, record_precision):
    """sfs_forward of the production configuration runs the fused persistent
    kernel (weights resident in shared memory): same bar as the unfused path."""
    from paper_2501_06377_gb300.surrogate import Surrogate, flat_from_reference
    P = S.init_params(C=PROD["channels"], M=PROD["modes"], L=PROD["blocks"], seed=4)
    P["Wd"] *= 50.0
    net = Surrogate(max_batch=4, **PROD)
    net.set_params(flat_from_reference(P, PROD["blocks"]))
    x, p, _ = _inputs(3, seed=5)
    out = torch_mod.empty((3, S.H, S.W), device="cuda")
    c0 = net.counters()
    net.forward(_cuda(torch_mod, x), _cuda(torch_mod, p), out)
    c1 = net.counters()
    # the fused path: no GEMM launch, a handful of kernels (rotation, image,
    # network, centring) instead of the unfused path's dozens
    assert c1["gemm_launches"] == c0["gemm_launches"]
    assert c1["kernel_launches"] - c0["kernel_launches"] <= 7
    xr = x.astype(np.float32).astype(np.float64)
    pr = p.astype(np.float32).astype(np.float64)
    ref = S.forward(P, xr, pr, L=PROD["blocks"], M=PROD["modes"])
    r = S.rotate(xr, S.rotation_angles(pr))
    got = out.cpu().numpy()
    corr_err = np.linalg.norm((got - r) - (ref - r)) / np.linalg.norm(ref - r)
    # flux-free correction: the output keeps each map's total flux
    A = S.cell_areas()[None, :, None]
    drift = np.abs((A * (got - xr)).sum(axis=(1, 2))) / (A * np.abs(xr)).sum(axis=(1, 2))
    record_precision("C5 surrogate forward (BF16 products, fused kernel) vs the FP64 reference",
                     None, None, float(drift.max()), correction_rel_l2=float(corr_err), correction_bar=1e-2)
    assert corr_err <= 1e-2, corr_err
    assert drift.max() <= 1e-6, drift


def test_fused_forward_follows_training_updates(torch_mod):
    """After AdamW steps the fused kernel's weight image is rebuilt: the loss of
    its output equals the loss the (unfused) training forward reports."""
    from paper_2501_06377_gb300.surrogate import Surrogate
    net = Surrogate(max_batch=4, seed=3, **PROD)
    x, p, y = _inputs(4, seed=7)
    xc, pc, yc = _cuda(torch_mod, x), _cuda(torch_mod, p), _cuda(torch_mod, y)
    out = torch_mod.empty_like(xc)
    net.forward(xc, pc, out)
    for _ in range(3):
        net.train_step(xc, pc, yc, 1e-3)
    net.forward(xc, pc, out)
    o = out.cpu().numpy().astype(np.float64)
    yy = y.astype(np.float32).astype(np.float64)
    loss_fused = float(np.mean(((o - yy) ** 2).sum(axis=(1, 2)) / (yy ** 2).sum(axis=(1, 2))))
    loss_train, _ = net.loss_grad(xc, pc, yc)
    assert loss_fused == pytest.approx(loss_train, rel=2e-3), (loss_fused, loss_train)
