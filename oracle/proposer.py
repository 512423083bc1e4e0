"""Oracle of the learned refinement proposer (plain numpy).

TEST INFRASTRUCTURE ONLY: used by the tests and the bench's CPU baseline; it
shares no code with the CUDA path.

The proposer has no counterpart in the paper: it stands in for the safety zone
of Section 2.1's refinement rule.  It is a 3-layer 3D convolutional net over the
block positions of every level (each level its own grid, zero padding at the
grid edge): 3 -> 16 -> 16 -> 1 channels, 3^3 kernels (cross-correlation:
out[co](x) = b[co] + sum_{ci,t} w[co][ci][t] * in[ci](x + t)), ReLU after the
first two layers.

Inference (``forward``): weights and every layer input are rounded to bfloat16
(round to nearest, ties to even); accumulation is exact here (float64).

Training (``loss_and_grad``, ``adam``; ``loss_and_grad_bf16`` adds the bfloat16
rounding points of the tensor-core path): the forward pass on the unrounded
master weights, the binary cross-entropy of the logits against next-step
flags over the positions of level >= 1 whose parent block exists, normalised
by a count given by the caller, its gradient by the chain rule through the
three layers (the adjoint of a zero-padded cross-correlation is the
correlation of the output gradient with the taps mirrored and the channel
roles swapped; the weight gradient correlates the output gradient with the
layer input), and the Adam update of Kingma and Ba (2015) with bias
correction.  Features and marking follow the definitions stated in
include/mrfv.h.
"""
from __future__ import annotations

import numpy as np

NWEIGHTS = 16 * 81 + 16 + 16 * 432 + 16 + 432 + 1


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


def unpack(blob: np.ndarray, dtype=np.float32):
    """The blob's weights and biases per layer: (W1 [16][3][27], B1 [16]), (W2
    [16][16][27], B2 [16]), (W3 [1][16][27], B3 [1]), as dtype."""
    b = np.asarray(blob, dtype=dtype)
    o = 0
    W1 = b[o:o + 16 * 81].reshape(16, 3, 27); o += 16 * 81
    B1 = b[o:o + 16]; o += 16
    W2 = b[o:o + 16 * 432].reshape(16, 16, 27); o += 16 * 432
    B2 = b[o:o + 16]; o += 16
    W3 = b[o:o + 432].reshape(1, 16, 27); o += 432
    B3 = b[o:o + 1]
    return (W1, B1), (W2, B2), (W3, B3)


def conv_level(x: np.ndarray, W: np.ndarray, bias: np.ndarray) -> np.ndarray:
    """x: [cin, nz, ny, nx] -> [cout, nz, ny, nx]; taps t = (dz+1)*9 + (dy+1)*3 + (dx+1)."""
    cin, nz, ny, nx = x.shape
    xp = np.zeros((cin, nz + 2, ny + 2, nx + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    out = np.zeros((W.shape[0], nz, ny, nx))
    for t in range(27):
        dz, dy, dx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
        sh = xp[:, 1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
        out += np.einsum("oc,czyx->ozyx", W[:, :, t].astype(np.float64), sh)
    return out + bias.astype(np.float64)[:, None, None, None]


def level_shapes(dim: int, levels: int, base_blocks):
    shapes = []
    for l in range(levels):
        n = [base_blocks[d] << l for d in range(dim)] + [1] * (3 - dim)
        shapes.append((n[2], n[1], n[0]))
    return shapes


def forward(blob: np.ndarray, feat: np.ndarray, shapes) -> np.ndarray:
    """feat: [3, positions] (levels concatenated) -> logits [positions]."""
    (W1, B1), (W2, B2), (W3, B3) = unpack(blob)
    W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    out = []
    off = 0
    for sh in shapes:
        n = int(np.prod(sh))
        x = bf16_round(feat[:, off:off + n]).reshape((3,) + sh).astype(np.float64)
        h = np.maximum(conv_level(x, W1, B1), 0.0)
        h = bf16_round(h.astype(np.float32)).astype(np.float64)
        h = np.maximum(conv_level(h, W2, B2), 0.0)
        h = bf16_round(h.astype(np.float32)).astype(np.float64)
        z = conv_level(h, W3, B3)
        out.append(z.reshape(-1))
        off += n
    return np.concatenate(out)


def features(dim: int, gamma: float, eps: float, levels_state, exist_maps, maxdet_maps, scale) -> np.ndarray:
    """Features [3, positions] from the dense level arrays ([nv][cells]), block maps,
    max normalised details and the analysis scales (s_rho, .., s_E)."""
    s_rho, s_p = scale[0], (gamma - 1.0) * scale[dim + 1]
    f0, f1, f2 = [], [], []
    for l, (q, ex, md) in enumerate(zip(levels_state, exist_maps, maxdet_maps)):
        rho = q[0]
        mom = q[1:1 + dim]
        E = q[dim + 1]
        p = (gamma - 1.0) * (E - 0.5 * np.sum(mom * mom, axis=0) / rho)
        bs = ex.shape
        a0 = np.zeros(bs); a1 = np.zeros(bs); a2 = np.zeros(bs)
        for idx in np.ndindex(*bs):
            if ex[idx]:
                sl = tuple(slice(8 * i, 8 * i + 8) for i in idx)
                a0[idx] = np.mean(np.nan_to_num(rho[sl])) / s_rho
                a1[idx] = np.mean(p[sl]) / s_p
                a2[idx] = min(md[idx] / eps, 8.0) / 8.0
            elif l > 0:
                par = tuple(i >> 1 for i in idx)
                if exist_maps[l - 1][par]:
                    sl = tuple(slice(8 * (i >> 1) + 4 * (i & 1), 8 * (i >> 1) + 4 * (i & 1) + 4) for i in idx)
                    qp = levels_state[l - 1]
                    rp = qp[0]
                    mp = qp[1:1 + dim]
                    pp = (gamma - 1.0) * (qp[dim + 1] - 0.5 * np.sum(mp * mp, axis=0) / rp)
                    a0[idx] = np.mean(rp[sl]) / s_rho
                    a1[idx] = np.mean(pp[sl]) / s_p
        f0.append(a0.ravel()); f1.append(a1.ravel()); f2.append(a2.ravel())
    return np.stack([np.concatenate(f0), np.concatenate(f1), np.concatenate(f2)])


# ----------------------------------------------------------------------------- training

def conv_level_input_grad(dy: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Adjoint of conv_level in its input: dy [cout, nz, ny, nx] -> dx [cin, nz, ny, nx],
    dx[ci](q) = sum_{co,t} W[co][ci][t] dy[co](q - t), dy zero outside the grid."""
    cout, nz, ny, nx = dy.shape
    dp = np.zeros((cout, nz + 2, ny + 2, nx + 2))
    dp[:, 1:-1, 1:-1, 1:-1] = dy
    dx = np.zeros((W.shape[1], nz, ny, nx))
    for t in range(27):
        dz, dyy, dxx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
        sh = dp[:, 1 - dz:1 - dz + nz, 1 - dyy:1 - dyy + ny, 1 - dxx:1 - dxx + nx]
        dx += np.einsum("oc,ozyx->czyx", W[:, :, t].astype(np.float64), sh)
    return dx


def conv_level_weight_grad(x: np.ndarray, dy: np.ndarray) -> np.ndarray:
    """Gradient of sum(dy * conv_level(x, W, b)) in W: [cout, cin, 27],
    dW[co][ci][t] = sum_p dy[co](p) x[ci](p + t), x zero outside the grid."""
    cin, nz, ny, nx = x.shape
    xp = np.zeros((cin, nz + 2, ny + 2, nx + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    dW = np.zeros((dy.shape[0], cin, 27))
    for t in range(27):
        dz, dyy, dxx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
        sh = xp[:, 1 + dz:1 + dz + nz, 1 + dyy:1 + dyy + ny, 1 + dxx:1 + dxx + nx]
        dW[:, :, t] = np.einsum("ozyx,czyx->oc", dy, sh)
    return dW


def parent_mask(shapes, exist_maps) -> np.ndarray:
    """Positions (levels concatenated) of level >= 1 whose parent block exists;
    exist_maps[l] has the level's block shape [nz, ny, nx] (or [ny, nx] in 2D)."""
    out = [np.zeros(int(np.prod(shapes[0])), dtype=bool)]
    for l in range(1, len(shapes)):
        nz, ny, nx = shapes[l]
        par = np.asarray(exist_maps[l - 1]).reshape(shapes[l - 1]).astype(bool)
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        out.append(par[z >> 1, y >> 1, x >> 1].reshape(-1))
    return np.concatenate(out)


def loss_and_grad(blob: np.ndarray, feats: np.ndarray, targets: np.ndarray, shapes, use: np.ndarray,
                  inv_count: float):
    """Binary cross-entropy with logits summed over the snapshots and over the
    positions where ``use`` holds and the target is not 255, times inv_count,
    and its gradient in the weights (the blob's order).  feats:
    [nsnap][3][positions], targets: [nsnap][positions] (0/1, 255 = left out).
    Master weights as given (no bfloat16 rounding), float64 throughout."""
    (W1, B1), (W2, B2), (W3, B3) = unpack(blob, np.float64)
    g = {k: 0.0 for k in ("W1", "B1", "W2", "B2", "W3", "B3")}
    loss = 0.0
    for f, y in zip(np.asarray(feats, dtype=np.float64), np.asarray(targets)):
        off = 0
        for sh in shapes:
            n = int(np.prod(sh))
            x = f[:, off:off + n].reshape((3,) + sh)
            u = use[off:off + n].reshape(sh) & (y[off:off + n].reshape(sh) != 255)
            yy = (y[off:off + n].reshape(sh) == 1).astype(np.float64)
            a1 = conv_level(x, W1, B1)
            h1 = np.maximum(a1, 0.0)
            a2 = conv_level(h1, W2, B2)
            h2 = np.maximum(a2, 0.0)
            z = conv_level(h2, W3, B3)[0]
            # BCE with logits: max(z, 0) - z y + log(1 + exp(-|z|)); dL/dz = sigmoid(z) - y
            lz = np.maximum(z, 0.0) - z * yy + np.log1p(np.exp(-np.abs(z)))
            loss += inv_count * float(np.sum(lz[u]))
            dz = np.where(u, (1.0 / (1.0 + np.exp(-z)) - yy) * inv_count, 0.0)[None]
            g["W3"] = g["W3"] + conv_level_weight_grad(h2, dz)
            g["B3"] = g["B3"] + dz.sum(axis=(1, 2, 3))
            d2 = conv_level_input_grad(dz, W3) * (a2 > 0)
            g["W2"] = g["W2"] + conv_level_weight_grad(h1, d2)
            g["B2"] = g["B2"] + d2.sum(axis=(1, 2, 3))
            d1 = conv_level_input_grad(d2, W2) * (a1 > 0)
            g["W1"] = g["W1"] + conv_level_weight_grad(x, d1)
            g["B1"] = g["B1"] + d1.sum(axis=(1, 2, 3))
            off += n
    grad = np.concatenate([np.broadcast_to(np.asarray(g[k], dtype=np.float64), s).ravel()
                           for k, s in (("W1", (16, 3, 27)), ("B1", (16,)), ("W2", (16, 16, 27)), ("B2", (16,)),
                                        ("W3", (1, 16, 27)), ("B3", (1,)))])
    return loss, grad


def _bf16_f64(x: np.ndarray) -> np.ndarray:
    """float64 -> float32 -> nearest bfloat16, returned as float64."""
    return bf16_round(np.asarray(x, dtype=np.float64).astype(np.float32)).astype(np.float64)


def loss_and_grad_bf16(blob: np.ndarray, feats: np.ndarray, targets: np.ndarray, shapes, use: np.ndarray,
                       inv_count: float, rnd=_bf16_f64):
    """The loss and gradient of training in bfloat16 (the tensor-core path): the
    forward pass of ``forward`` (weights, features and hidden activations rounded
    by ``rnd``), dL/dz of the binary cross-entropy (positions where ``use`` holds
    and the target is not 255), the gradients of the layer inputs through the
    rounded weights, masked by the ReLU and rounded by ``rnd`` (dL/dz itself is
    rounded before it enters the layer-3 input gradient), and the weight
    gradients as products of those rounded operands, accumulated exactly.  With
    ``rnd`` the identity this is ``loss_and_grad``."""
    (W1, B1), (W2, B2), (W3, B3) = unpack(blob, np.float64)
    W1b, W2b, W3b = rnd(W1), rnd(W2), rnd(W3)
    g = {k: 0.0 for k in ("W1", "B1", "W2", "B2", "W3", "B3")}
    loss = 0.0
    for f, y in zip(np.asarray(feats, dtype=np.float64), np.asarray(targets)):
        off = 0
        for sh in shapes:
            n = int(np.prod(sh))
            x = rnd(f[:, off:off + n]).reshape((3,) + sh)
            u = use[off:off + n].reshape(sh) & (y[off:off + n].reshape(sh) != 255)
            yy = (y[off:off + n].reshape(sh) == 1).astype(np.float64)
            h1 = rnd(np.maximum(conv_level(x, W1b, B1), 0.0))
            h2 = rnd(np.maximum(conv_level(h1, W2b, B2), 0.0))
            z = conv_level(h2, W3b, B3)[0]
            lz = np.maximum(z, 0.0) - z * yy + np.log1p(np.exp(-np.abs(z)))
            loss += inv_count * float(np.sum(lz[u]))
            dz = np.where(u, (1.0 / (1.0 + np.exp(-z)) - yy) * inv_count, 0.0)[None]
            dzf = dz.astype(np.float32).astype(np.float64) if rnd is _bf16_f64 else dz
            g["W3"] = g["W3"] + conv_level_weight_grad(h2, dzf)
            g["B3"] = g["B3"] + dzf.sum(axis=(1, 2, 3))
            d2 = rnd(conv_level_input_grad(rnd(dzf), W3b) * (h2 > 0))
            g["W2"] = g["W2"] + conv_level_weight_grad(h1, d2)
            g["B2"] = g["B2"] + d2.sum(axis=(1, 2, 3))
            d1 = rnd(conv_level_input_grad(d2, W2b) * (h1 > 0))
            g["W1"] = g["W1"] + conv_level_weight_grad(x, d1)
            g["B1"] = g["B1"] + d1.sum(axis=(1, 2, 3))
            off += n
    grad = np.concatenate([np.broadcast_to(np.asarray(g[k], dtype=np.float64), s).ravel()
                           for k, s in (("W1", (16, 3, 27)), ("B1", (16,)), ("W2", (16, 16, 27)), ("B2", (16,)),
                                        ("W3", (1, 16, 27)), ("B3", (1,)))])
    return loss, grad


def adam(w: np.ndarray, grad: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, lr: float,
         beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam step (t >= 1): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
    w <- w - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).  Returns (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
