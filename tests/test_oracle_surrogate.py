"""Pins for the FP64 reference of the learned surrogate (oracle/surrogate_ref.py).

The rotation layer is pinned by exact integer shifts (np.roll), the DFT
pair by band-limited reconstruction, the hand-written backward pass by
central finite differences of the loss, and AdamW by its first-step closed
form.
"""
import math

import numpy as np
import pytest

import oracle.surrogate_ref as S


def test_dft_pair_reconstructs_band_limited_rows():
    n, m = 128, 24
    F, Gm = S.dft_mats(n, m)
    rng = np.random.default_rng(0)
    coef = rng.normal(size=(2, m))
    coef[1, 0] = 0.0
    l = np.arange(n)
    sig = sum(coef[0, k] * np.cos(2 * math.pi * k * l / n) + coef[1, k] * np.sin(2 * math.pi * k * l / n)
              for k in range(m))
    np.testing.assert_allclose(Gm @ (F @ sig), sig, atol=1e-12)


def test_rotation_by_whole_cells_is_a_roll():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, S.H, S.W))
    for cells in (1, 5, -3):
        alpha = np.full((2, S.H), 2 * math.pi * cells / S.W)
        np.testing.assert_allclose(S.rotate(x, alpha), np.roll(x, cells, axis=2), atol=1e-10)


def test_rotation_angles_follow_the_rotation_profile():
    p = np.array([[13.38, -2.30, -1.62, 15.0, 500.0]])
    a = S.rotation_angles(p)[0]
    frame = 360.0 / 27.2753
    s2 = math.cos(S.H // 2 * math.pi / (S.H - 1)) ** 2   # row next to the equator
    assert a[S.H // 2] == pytest.approx(math.radians(13.38 - 2.30 * s2 - 1.62 * s2 * s2 - frame), rel=1e-12)
    assert a[0] == pytest.approx(math.radians(13.38 - 2.30 - 1.62 - frame), rel=1e-12)  # pole


def _tiny():
    C, M, L = 8, 4, 1
    P = S.init_params(C=C, M=M, L=L, seed=3)
    rng = np.random.default_rng(4)
    x = rng.normal(0, 50.0, (2, S.H, S.W))
    y = x + rng.normal(0, 5.0, (2, S.H, S.W))
    p = np.array([[13.0, -2.1, -1.7, 12.0, 400.0], [13.9, -2.5, -1.5, 18.0, 650.0]])
    return P, x, y, p, C, M, L


def test_backward_matches_central_differences():
    P, x, y, p, C, M, L = _tiny()
    loss, g = S.loss_and_grad(P, x, p, y, L=L, M=M)
    rng = np.random.default_rng(5)
    for name in P:
        flat = P[name].reshape(-1)
        nz = np.flatnonzero(np.abs(g[name].reshape(-1)) > 0)
        picks = rng.choice(nz, size=min(3, nz.size), replace=False) if nz.size else []
        for i in picks:
            h = 1e-3 * max(1.0, abs(flat[i]))   # O(h^2) truncation, far above roundoff
            old = flat[i]
            flat[i] = old + h
            lp, _ = S.loss_and_grad(P, x, p, y, L=L, M=M)
            flat[i] = old - h
            lm, _ = S.loss_and_grad(P, x, p, y, L=L, M=M)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert g[name].reshape(-1)[i] == pytest.approx(fd, rel=1e-5, abs=1e-12), (name, i)


def test_adamw_first_step_closed_form():
    P = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.3, -0.1, 0.0])}
    m = {"a": np.zeros(3)}
    v = {"a": np.zeros(3)}
    lr, wd = 1e-2, 0.1
    P, m, v = S.adamw_step(P, g, m, v, 1, lr, wd=wd)
    expect = np.array([1.0, -2.0, 0.5]) - lr * (np.array([1.0, -1.0, 0.0]) * np.array([0.3, 0.1, 0.0])
                                                / (np.array([0.3, 0.1, 0.0]) + 1e-8)
                                                + wd * np.array([1.0, -2.0, 0.5]))
    np.testing.assert_allclose(P["a"], expect, rtol=1e-7)


def test_parameter_count_is_about_two_million():
    assert 1.6e6 < S.n_params(S.init_params()) < 2.4e6


def test_output_keeps_the_total_flux_of_the_input():
    """x_next = r + s (delta - <delta>_A): the correction has no net flux and
    the rotation keeps every row's sum, so sum A x_next = sum A x."""
    P, x, y, p, C, M, L = _tiny()
    P["Wd"] *= 300.0
    P["bd"][:] = 0.7
    xn = S.forward(P, x, p, L=L, M=M)
    A = S.cell_areas()[None, :, None]
    tot = (A * x).sum(axis=(1, 2))
    scale = (A * np.abs(x)).sum(axis=(1, 2))
    np.testing.assert_allclose((A * xn).sum(axis=(1, 2)), tot, rtol=0, atol=1e-12 * scale.max())
    assert np.abs(xn - S.rotate(x, S.rotation_angles(p))).max() > 1.0   # the correction is not zero
