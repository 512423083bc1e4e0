"""Oracle of the learned refinement proposer (plain numpy).

TEST INFRASTRUCTURE ONLY: used by the tests and the bench's CPU baseline; it
shares no code with the CUDA path.

The proposer is a 3-layer 3D convolutional net over the block positions of every
level (each level its own grid, zero padding at the grid edge): 3 -> 16 -> 16 -> 1
channels, 3^3 kernels (cross-correlation: out[co](x) = b[co] + sum_{ci,t}
w[co][ci][t] * in[ci](x + t)), ReLU after the first two layers.  Weights and
every layer input are rounded to bfloat16 (round to nearest, ties to even),
accumulation is exact here (float64).  Features and marking follow the
definitions stated in include/mrfv.h.
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


def unpack(blob: np.ndarray):
    b = np.asarray(blob, dtype=np.float32)
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
