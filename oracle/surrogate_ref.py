"""FP64 numpy reference of the learned one-day surrogate (forward + backward).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the GPU surrogate's
forward pass, gradients and optimizer step are checked against this plain
restatement, and this file's own backward pass is checked against central
finite differences.

The paper has no learned component (it only mentions a PINN-based SFT in its
introduction); the network follows the build's specification: a neural
operator on 256 x 512 maps, conditioned on the five flow/diffusion
parameters, that proposes one-day advances.

Network (maps x [B, H, W], parameters p [B, 5], all names as in the GPU code):
  R:      r = per-row rotation of x in phi by the day's differential
          rotation angle alpha_j(p) (exact in phi-Fourier space, fixed, no
          weights): X = x F, X_k *= exp(-i k alpha_j), r = X G.
  embed:  4x4 patches of [x/s, r/s] (32 values) + p (5) + cos/sin of the
          patch-row colatitude (2), zero-padded to 48 -> h = E We + be   (C)
  block:  spectral mixing along phi of every latent row i (per channel):
            Hh = Fm h_i (2M x C, M modes),  Yh = w_i (.) Hh (complex, per
            (i, k, c)),  u = h + Gm Yh;
          channel MLP: z = u W1 + b1, a = gelu(z), h = u + a W2 + b2
  decode: d = h Wd + bd (16 per patch) -> delta [B, H, W] (unpatchify)
  output: x_next = r + s * (delta - <delta>_A), <.>_A the area-weighted mean
          over the sphere (the grid's cell areas, polar caps included), so
          the correction carries no net flux and x_next keeps the total
          flux of r, which keeps that of x (a phi rotation keeps row sums)
  loss:   mean_b ||x_next - y||^2 / ||y||^2   (relative MSE)
"""
from __future__ import annotations

import math

import numpy as np

H, W = 256, 512
PATCH = 4
HT, WT = H // PATCH, W // PATCH          # 64 x 128 latent tokens
KE = 48                                   # embed input features (39 used, zero-padded)
SCALE_G = 100.0                           # map normalisation (G)
DT_H = 24.0                               # one day


def gelu(z):
    """tanh-form GELU (Hendrycks & Gimpel 2016)."""
    return 0.5 * z * (1.0 + np.tanh(math.sqrt(2.0 / math.pi) * (z + 0.044715 * z**3)))


def gelu_grad(z):
    c = math.sqrt(2.0 / math.pi)
    t = np.tanh(c * (z + 0.044715 * z**3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * c * (1.0 + 3 * 0.044715 * z * z)


def dft_mats(n, m):
    """Real DFT of length n truncated to modes 0..m-1: F [2m, n] (rows: cos
    parts then -sin parts) and its pseudo-inverse synthesis G [n, 2m]
    (weights 1/n for k = 0 and k = n/2, 2/n otherwise)."""
    l = np.arange(n)
    k = np.arange(m)
    ang = 2.0 * math.pi * np.outer(k, l) / n
    F = np.concatenate([np.cos(ang), -np.sin(ang)], axis=0)
    wgt = np.where((k == 0) | (2 * k == n), 1.0 / n, 2.0 / n)
    Gm = np.concatenate([(wgt[:, None] * np.cos(ang)).T, -(wgt[:, None] * np.sin(ang)).T], axis=1)
    return F, Gm


def cell_areas():
    """Area weight of one stored entry of row j (poles: the cap shared over
    its W entries), the grid convention of the solver."""
    dth, dph = math.pi / (H - 1), 2.0 * math.pi / W
    a = np.sin(np.arange(H) * dth) * dth * dph
    a[0] = a[-1] = 2.0 * math.pi * (1.0 - math.cos(0.5 * dth)) / W
    return a


def rotation_angles(p_phys):
    """alpha[b, j] (rad): the day's rotation of row j relative to the frame,
    from the physical parameters (o0, o2, o4 deg/day, U m/s, eta km^2/s);
    Omega(lat) = o0 + o2 sin^2 lat + o4 sin^4 lat - 360/27.2753."""
    theta = np.arange(H) * (math.pi / (H - 1))
    s2 = np.cos(theta) ** 2
    frame = 360.0 / 27.2753
    om = (p_phys[:, 0:1] + p_phys[:, 1:2] * s2[None, :] + p_phys[:, 2:3] * s2[None, :] ** 2) - frame
    return np.radians(om) * (DT_H / 24.0)


def rotate(x, alpha):
    """Layer R: r[b, j, :] = x[b, j, :] shifted by alpha[b, j] in phi
    (exact for band-limited rows; all W/2+1 modes kept)."""
    F, Gm = dft_mats(W, W // 2 + 1)
    M = W // 2 + 1
    X = x @ F.T                                   # [B, H, 2M]
    k = np.arange(M)
    c = np.cos(k[None, None, :] * alpha[:, :, None])
    s = np.sin(k[None, None, :] * alpha[:, :, None])
    re, im = X[..., :M], X[..., M:]
    # multiply by exp(-i k alpha)
    Y = np.concatenate([re * c + im * s, im * c - re * s], axis=-1)
    return Y @ Gm.T


def normalise_params(p_phys):
    """The five conditioning parameters mapped to about [-1, 1]."""
    ref = np.array([13.38, -2.30, -1.62, 15.0, 500.0])
    spread = np.array([1.338, 0.230, 0.162, 5.0, 250.0])
    return (p_phys - ref) / spread


def init_params(C=128, M=24, L=4, seed=0):
    rng = np.random.default_rng(seed)
    P = {"We": rng.normal(0, 1 / math.sqrt(39), (KE, C)), "be": np.zeros(C),
         "Wd": rng.normal(0, 0.02 / math.sqrt(C), (C, PATCH * PATCH)), "bd": np.zeros(PATCH * PATCH)}
    P["We"][39:] = 0.0
    for l in range(L):
        P["w%d" % l] = np.concatenate([np.ones((HT, M, C, 1)), np.zeros((HT, M, C, 1))], -1) * 0.5 \
            + rng.normal(0, 0.02, (HT, M, C, 2))
        P["W1_%d" % l] = rng.normal(0, 1 / math.sqrt(C), (C, 2 * C))
        P["b1_%d" % l] = np.zeros(2 * C)
        P["W2_%d" % l] = rng.normal(0, 0.5 / math.sqrt(2 * C), (2 * C, C))
        P["b2_%d" % l] = np.zeros(C)
    return P


def patchify(img):
    """[B, H, W] -> [B, HT, WT, 16] (row-major 4x4 patches)."""
    B = img.shape[0]
    return img.reshape(B, HT, PATCH, WT, PATCH).transpose(0, 1, 3, 2, 4).reshape(B, HT, WT, PATCH * PATCH)


def unpatchify(t):
    B = t.shape[0]
    return t.reshape(B, HT, WT, PATCH, PATCH).transpose(0, 1, 3, 2, 4).reshape(B, H, W)


def embed_inputs(x, r, pn):
    """E [B, HT, WT, 48]."""
    B = x.shape[0]
    E = np.zeros((B, HT, WT, KE))
    E[..., 0:16] = patchify(x / SCALE_G)
    E[..., 16:32] = patchify(r / SCALE_G)
    E[..., 32:37] = pn[:, None, None, :]
    th = (np.arange(HT) + 0.5) * PATCH * (math.pi / (H - 1))
    E[..., 37] = np.cos(th)[None, :, None]
    E[..., 38] = np.sin(th)[None, :, None]
    return E


def forward(P, x, p_phys, L=4, M=24, keep=False):
    """x_next [B, H, W]; with keep=True also the activations for backward."""
    alpha = rotation_angles(p_phys)
    r = rotate(x, alpha)
    E = embed_inputs(x, r, normalise_params(p_phys))
    F, Gm = dft_mats(WT, M)
    h = E @ P["We"] + P["be"]                       # [B, HT, WT, C]
    acts = {"E": E, "r": r, "blocks": []}
    for l in range(L):
        w = P["w%d" % l]
        Hh = np.einsum("kl,bilc->bikc", F, h)        # [B, HT, 2M, C]
        hr, hi = Hh[:, :, :M], Hh[:, :, M:]
        wr, wi = w[..., 0][None], w[..., 1][None]
        Yh = np.concatenate([wr * hr - wi * hi, wr * hi + wi * hr], axis=2)
        u = h + np.einsum("lk,bikc->bilc", Gm, Yh)
        z = u @ P["W1_%d" % l] + P["b1_%d" % l]
        a = gelu(z)
        hn = u + a @ P["W2_%d" % l] + P["b2_%d" % l]
        acts["blocks"].append({"h": h, "Hh": Hh, "u": u, "z": z, "a": a})
        h = hn
    d = h @ P["Wd"] + P["bd"]
    acts["hL"] = h
    dmap = unpatchify(d)
    Ar = cell_areas()[None, :, None]
    mean = (Ar * dmap).sum(axis=(1, 2)) / (Ar.sum() * W)
    xn = r + SCALE_G * (dmap - mean[:, None, None])
    return (xn, acts) if keep else xn


def loss_and_grad(P, x, p_phys, y, L=4, M=24):
    """Relative-MSE loss and its gradient for every parameter."""
    xn, A = forward(P, x, p_phys, L, M, keep=True)
    B = x.shape[0]
    den = (y**2).sum(axis=(1, 2))
    diff = xn - y
    loss = float(((diff**2).sum(axis=(1, 2)) / den).mean())
    dxn = 2.0 * diff / den[:, None, None] / B
    g = {}
    Ar = cell_areas()[None, :, None]
    gsum = dxn.sum(axis=(1, 2))
    dd = patchify(SCALE_G * (dxn - Ar * gsum[:, None, None] / (Ar.sum() * W)))   # [B, HT, WT, 16]
    hL = A["hL"]
    g["Wd"] = np.einsum("bijc,bijo->co", hL, dd)
    g["bd"] = dd.sum(axis=(0, 1, 2))
    dh = dd @ P["Wd"].T
    F, Gm = dft_mats(WT, M)
    for l in reversed(range(L)):
        blk = A["blocks"][l]
        du = dh.copy()
        g["W2_%d" % l] = np.einsum("bijc,bijo->co", blk["a"], dh)
        g["b2_%d" % l] = dh.sum(axis=(0, 1, 2))
        da = dh @ P["W2_%d" % l].T
        dz = da * gelu_grad(blk["z"])
        g["W1_%d" % l] = np.einsum("bijc,bijo->co", blk["u"], dz)
        g["b1_%d" % l] = dz.sum(axis=(0, 1, 2))
        du += dz @ P["W1_%d" % l].T
        dYh = np.einsum("lk,bilc->bikc", Gm, du)     # Gm^T du
        w = P["w%d" % l]
        hr, hi = blk["Hh"][:, :, :M], blk["Hh"][:, :, M:]
        dyr, dyi = dYh[:, :, :M], dYh[:, :, M:]
        gw = np.zeros_like(w)
        gw[..., 0] = (dyr * hr + dyi * hi).sum(0)
        gw[..., 1] = (-dyr * hi + dyi * hr).sum(0)
        g["w%d" % l] = gw
        wr, wi = w[..., 0][None], w[..., 1][None]
        dHh = np.concatenate([wr * dyr + wi * dyi, -wi * dyr + wr * dyi], axis=2)
        dh = du + np.einsum("kl,bikc->bilc", F, dHh)  # F^T dHh
    g["We"] = np.einsum("bijc,bijo->co", A["E"], dh)
    g["be"] = dh.sum(axis=(0, 1, 2))
    return loss, g


def adamw_step(P, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
    """Decoupled weight decay Adam (Loshchilov & Hutter 2019), in place."""
    for k in P:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] ** 2
        mh = m[k] / (1 - beta1**t)
        vh = v[k] / (1 - beta2**t)
        P[k] = P[k] - lr * (mh / (np.sqrt(vh) + eps) + wd * P[k])
    return P, m, v


def n_params(P):
    return int(sum(v.size for v in P.values()))
