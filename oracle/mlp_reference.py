"""Plain numpy reference of the surrogate network (test infrastructure only).

Network: Fourier features [sin(2 pi F u), cos(2 pi F u)] of u = (r - c)/R
(32 frequencies), four hidden layers of 256 with SiLU, one linear output;
loss mean((y - t)^2).  Forward and the analytic backward pass are written out
in FP64; with bf16=True the values are rounded to bfloat16 (round to nearest
even) wherever the GPU kernels store BF16 (features, hidden activations,
weights used by the matrix products, gradients flowing backward), so the GPU
gradients can be compared term by term.  The FP64 version is pinned by
finite differences in the tests.

Flat parameter layout: W1[256x64] b1[256] W2[256x256] b2 W3 b3 W4 b4 w5[256] b5.
"""
import numpy as np

HIDDEN = 256
FEAT = 64
LAYERS = 4


def layout():
    off = 0
    spec = []
    for l in range(LAYERS):
        kin = FEAT if l == 0 else HIDDEN
        spec.append(("W%d" % (l + 1), off, (HIDDEN, kin)))
        off += HIDDEN * kin
        spec.append(("b%d" % (l + 1), off, (HIDDEN,)))
        off += HIDDEN
    spec.append(("w5", off, (HIDDEN,)))
    off += HIDDEN
    spec.append(("b5", off, ()))
    off += 1
    return spec, off


def unpack(flat):
    spec, total = layout()
    assert flat.size == total
    out = {}
    for name, off, shape in spec:
        n = int(np.prod(shape)) if shape else 1
        v = flat[off:off + n].astype(np.float64)
        out[name] = v.reshape(shape) if shape else v[0]
    return out


def pack(d):
    spec, total = layout()
    flat = np.zeros(total)
    for name, off, shape in spec:
        n = int(np.prod(shape)) if shape else 1
        flat[off:off + n] = np.asarray(d[name], np.float64).reshape(-1)
    return flat


def bf16(x):
    """Round float64/float32 values to bfloat16 (nearest, ties to even), as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def features(freq, centre, inv_r, pos):
    u = (np.asarray(pos, np.float64) - np.asarray(centre)) * inv_r
    ph = 2.0 * np.pi * u @ np.asarray(freq, np.float64).T
    return np.concatenate([np.sin(ph), np.cos(ph)], axis=1)


def forward(flat, freq, centre, inv_r, pos, use_bf16=False):
    p = unpack(flat)
    r = bf16 if use_bf16 else (lambda x: np.asarray(x, np.float64))
    X = r(features(freq, centre, inv_r, pos))
    H, Z = [X], []
    for l in range(LAYERS):
        z = H[-1] @ r(p["W%d" % (l + 1)]).T + p["b%d" % (l + 1)]
        Z.append(z)
        H.append(r(silu(z)))
    y = H[-1] @ p["w5"] + p["b5"]
    return y, (p, H, Z)


def loss_and_grad(flat, freq, centre, inv_r, pos, t, use_bf16=False):
    """(loss, flat gradient) of mean((y - t)^2)."""
    r = bf16 if use_bf16 else (lambda x: np.asarray(x, np.float64))
    y, (p, H, Z) = forward(flat, freq, centre, inv_r, pos, use_bf16)
    n = y.size
    dy = 2.0 * (y - t) / n
    g = {"w5": H[-1].T @ dy, "b5": dy.sum()}
    dZ = r(np.outer(dy, p["w5"]) * silu_grad(Z[-1]))
    for l in range(LAYERS - 1, -1, -1):
        g["W%d" % (l + 1)] = dZ.T @ H[l]
        g["b%d" % (l + 1)] = dZ.sum(axis=0)
        if l > 0:
            dZ = r((dZ @ r(p["W%d" % (l + 1)])) * silu_grad(Z[l - 1]))
    return float(np.mean((y - t) ** 2)), pack(g)
