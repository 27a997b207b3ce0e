"""FP64 reference of the learned multigrid correction network (spec extension).

TEST INFRASTRUCTURE ONLY: used by tests and the training-data generator, never by the
library.  Plain numpy, FP64, written from the definition:

  network  y = W3 * relu(W2 * relu(W1 * x + b1) + b2) + b3
  where `*` is a 3x3x3 convolution with zero padding (the zero Dirichlet wall) on the
  interior grid, channels 1 -> 16 -> 16 -> 1.  Input x = D^-1 r, the residual of the
  sub-step operator (I - c Lap_h) scaled by its diagonal D = 1 + 6 c / h^2; output y is
  added to the multigrid correction e; target t = e* - e, the exact remaining error.

  Loss, per sample with its own kappa: 0.5 * mean((Ahat^p (y - t))^2), where
  Ahat = D^-1 (I - c Lap_h) = I - kappa N, N the sum over the 6 face neighbours (zero
  walls) and kappa = (c/h^2) / (1 + 6 c/h^2).  p = 0 is the plain error norm; p = 1 the
  scaled residual left after adding y (Ahat t = x); p = 2 weights each error mode by
  the square of its eigenvalue of Ahat, i.e. it ignores smooth modes (eigenvalues near
  0), which the coarse-grid correction removes, and measures the oscillatory modes a
  smoother must damp.  kappa = 0 reduces every p to the plain error norm.

Array conventions: grid functions [z][y][x]; activations [C][z][y][x]; weights
W[c_out][tap][c_in] with tap = (dz+1)*9 + (dy+1)*3 + (dx+1), offsets in {-1, 0, 1}.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
CH = 16


def shift(a: np.ndarray, d) -> np.ndarray:
    """b[..., z, y, x] = a[..., z+dz, y+dy, x+dx], zero outside the grid."""
    dz, dy, dx = d
    out = np.zeros_like(a)
    n = a.shape[-1]

    def sl(o):
        return slice(max(0, -o), n - max(0, o)), slice(max(0, o), n - max(0, -o))

    (oz, iz), (oy, iy), (ox, ix) = sl(dz), sl(dy), sl(dx)
    out[..., oz, oy, ox] = a[..., iz, iy, ix]
    return out


def conv(a: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """a: [Cin][n][n][n], W: [Cout][27][Cin], b: [Cout] -> [Cout][n][n][n]."""
    out = np.zeros((W.shape[0],) + a.shape[1:])
    for t, d in enumerate(TAPS):
        out += np.einsum("oc,czyx->ozyx", W[:, t, :], shift(a, d))
    return out + b[:, None, None, None]


def conv_input_grad(g: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Gradient of sum(g * conv(a, W, b)) with respect to a: a transposed convolution."""
    out = np.zeros((W.shape[2],) + g.shape[1:])
    for t, (dz, dy, dx) in enumerate(TAPS):
        out += np.einsum("oc,ozyx->czyx", W[:, t, :], shift(g, (-dz, -dy, -dx)))
    return out


def conv_weight_grad(g: np.ndarray, a: np.ndarray) -> np.ndarray:
    """Gradient of sum(g * conv(a, W, b)) with respect to W: [Cout][27][Cin]."""
    Wg = np.zeros((g.shape[0], 27, a.shape[0]))
    for t, d in enumerate(TAPS):
        Wg[:, t, :] = np.einsum("ozyx,czyx->oc", g, shift(a, d))
    return Wg


def apply_ahat(v: np.ndarray, kappa: float) -> np.ndarray:
    """Ahat v = v - kappa * (sum of the 6 face neighbours of v), zero outside the grid."""
    nb = np.zeros_like(v)
    for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        nb += shift(v, d)
    return v - kappa * nb


def init_params(seed: int = 5, ch: int = CH) -> dict:
    """He-scaled random weights, zero biases."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((ch, 27, 1)) * np.sqrt(2.0 / 27),
        "b1": np.zeros(ch),
        "W2": rng.standard_normal((ch, 27, ch)) * np.sqrt(2.0 / (27 * ch)),
        "b2": np.zeros(ch),
        "W3": rng.standard_normal((1, 27, ch)) * np.sqrt(1.0 / (27 * ch)),
        "b3": np.zeros(1),
    }


def forward(p: dict, x: np.ndarray):
    """x: [n][n][n] -> (y [n][n][n], cache)."""
    x4 = x[None]
    z1 = conv(x4, p["W1"], p["b1"])
    a1 = np.maximum(z1, 0.0)
    z2 = conv(a1, p["W2"], p["b2"])
    a2 = np.maximum(z2, 0.0)
    y = conv(a2, p["W3"], p["b3"])[0]
    return y, (x4, z1, a1, z2, a2)


def loss_and_grads(p: dict, xs, ts, kappas=None, power: int = 1):
    """Mean over all points of all samples of 0.5 (Ahat_kappa^power (y - t))^2 (kappa = 0
    for every sample when kappas is None), and its parameter gradients."""
    npts = sum(x.size for x in xs)
    if kappas is None:
        kappas = [0.0] * len(xs)
    L = 0.0
    g = {k: np.zeros_like(v) for k, v in p.items()}
    for x, t, kap in zip(xs, ts, kappas):
        y, (x4, z1, a1, z2, a2) = forward(p, x)
        w = y - t
        for _ in range(power):
            w = apply_ahat(w, kap)
        L += 0.5 * float((w * w).sum()) / npts
        gy = w / npts
        for _ in range(power):  # Ahat is symmetric
            gy = apply_ahat(gy, kap)
        gy = gy[None]
        g["W3"] += conv_weight_grad(gy, a2)
        g["b3"] += gy.sum(axis=(1, 2, 3))
        gz2 = conv_input_grad(gy, p["W3"]) * (z2 > 0)
        g["W2"] += conv_weight_grad(gz2, a1)
        g["b2"] += gz2.sum(axis=(1, 2, 3))
        gz1 = conv_input_grad(gz2, p["W2"]) * (z1 > 0)
        g["W1"] += conv_weight_grad(gz1, x4)
        g["b1"] += gz1.sum(axis=(1, 2, 3))
    return L, g


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round FP64 values to the nearest BF16 value (round half to even)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
