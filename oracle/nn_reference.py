"""FP64 numpy reference of the learned warm start's network (test infrastructure only).

TEST INFRASTRUCTURE ONLY: only the test suite and the smoke check use this module; the product
path runs the CUDA kernels of the library.  It shares no code with them.

The network maps (solid mask, signed distance, log Kn n1) to scaled (rho', u1, u2, u3) on a periodic
grid: a U-Net with L levels and C_l = C 2^l channels at level l, 3 x 3 x 3 periodic convolutions
with biases, ReLU, 2 x 2 x 2 mean pooling and nearest-neighbour upsampling:

    encoder level l:   h = relu(conv(h, e_l_a)); h = relu(conv(h, e_l_b)); keep h, pool (l < L-1)
    decoder level l:   h = concat(kept_l, up(h)); h = relu(conv(h, d_l_a)); h = relu(conv(h, d_l_b))
    output:            y = conv(h, out)

Parameters are an ordered list of (w [co][ci][27], b [co]) in the order e_0_a, e_0_b, ...,
e_{L-1}_b, d_{L-2}_a, d_{L-2}_b, ..., d_0_b, out.  Tap k = (kz * 3 + ky) * 3 + kx reads the input at
offset (kz - 1, ky - 1, kx - 1).  Tensors are [c][z][y][x].
"""
import numpy as np


def _offsets():
    return [(k // 9 - 1, (k // 3) % 3 - 1, k % 3 - 1) for k in range(27)]


def shifted(x, off):
    """x[c][z + dz][y + dy][x + dx] with periodic wrap."""
    dz, dy, dx = off
    return np.roll(x, shift=(-dz, -dy, -dx), axis=(1, 2, 3))


def conv3d(x, w, b=None):
    y = np.zeros((w.shape[0],) + x.shape[1:])
    for k, off in enumerate(_offsets()):
        y += np.einsum("oc,czyx->ozyx", w[:, :, k], shifted(x, off))
    if b is not None:
        y += b[:, None, None, None]
    return y


def conv3d_dgrad(dy, w):
    """Gradient with respect to the input of y = conv3d(x, w)."""
    dx = np.zeros((w.shape[1],) + dy.shape[1:])
    for k, (dz, dyy, dxx) in enumerate(_offsets()):
        dx += np.einsum("oc,ozyx->czyx", w[:, :, k], shifted(dy, (-dz, -dyy, -dxx)))
    return dx


def conv3d_wgrad(x, dy):
    """Gradients with respect to w and b of y = conv3d(x, w) + b."""
    dw = np.zeros((dy.shape[0], x.shape[0], 27))
    for k, off in enumerate(_offsets()):
        dw[:, :, k] = np.einsum("ozyx,czyx->oc", dy, shifted(x, off))
    return dw, dy.sum(axis=(1, 2, 3))


def pool2(x):
    c, d, h, w = x.shape
    return x.reshape(c, d // 2, 2, h // 2, 2, w // 2, 2).mean(axis=(2, 4, 6))


def pool2_bwd(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up2_bwd(dy):
    c, d, h, w = dy.shape
    return dy.reshape(c, d // 2, 2, h // 2, 2, w // 2, 2).sum(axis=(2, 4, 6))


def layer_shapes(levels, base, cin, cout):
    """(ci, co) of every convolution in parameter order."""
    ch = [base * 2 ** l for l in range(levels)]
    shapes = []
    for l in range(levels):
        shapes.append((cin if l == 0 else ch[l - 1], ch[l]))
        shapes.append((ch[l], ch[l]))
    for l in reversed(range(levels - 1)):
        shapes.append((ch[l] + ch[l + 1], ch[l]))
        shapes.append((ch[l], ch[l]))
    shapes.append((ch[0], cout))
    return shapes


def round_bf16(a):
    """The values a float32 tensor would carry after rounding to bfloat16 (round to nearest even),
    as float64: the operands of a BF16 tensor-core product."""
    u = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def forward(params, x, levels, bf16_operands=False):
    """Returns (y, cache) with the activations the backward pass needs.  bf16_operands: every
    convolution reads its input rounded to bfloat16 (the weights are expected BF16-representable
    already), as a BF16 tensor-core convolution with FP32 accumulation does."""
    rb = round_bf16 if bf16_operands else (lambda t: t)
    cache = []
    kept = []
    h = x
    p = 0
    for l in range(levels):
        for _ in range(2):
            w, b = params[p]
            a = np.maximum(conv3d(rb(h), w, b), 0.0)
            cache.append(("conv_relu", h, a))
            h = a
            p += 1
        if l < levels - 1:
            kept.append(h)
            cache.append(("pool", h.shape))
            h = pool2(h)
    for l in reversed(range(levels - 1)):
        u = up2(h)
        cache.append(("up", kept[l].shape[0]))
        h = np.concatenate([kept[l], u], axis=0)
        for _ in range(2):
            w, b = params[p]
            a = np.maximum(conv3d(rb(h), w, b), 0.0)
            cache.append(("conv_relu", h, a))
            h = a
            p += 1
    w, b = params[p]
    y = conv3d(rb(h), w, b)
    cache.append(("conv", h))
    return y, cache


def masked_mse(y, t, mask):
    """sum over channels and fluid voxels of (y - t)^2 / (channels x fluid voxels), and dL/dy."""
    m = mask[None].astype(np.float64)
    count = y.shape[0] * max(float(mask.sum()), 1.0)
    r = m * (y - t)
    return float((r * r).sum() / count), 2.0 * r / count


def _wgrad(x, dy, rb):
    """(dw, db) with dw from the rounded operands rb(x), rb(dy) and db from dy itself."""
    dw, _ = conv3d_wgrad(rb(x), rb(dy))
    return dw, dy.sum(axis=(1, 2, 3))


def backward(params, cache, dy, levels, bf16_operands=False):
    """Gradients [(dw, db)] in parameter order for the output gradient dy.  bf16_operands: every
    data gradient reads its input gradient rounded to bfloat16, and every weight gradient reads the
    layer input and the output gradient rounded to bfloat16 (the operands of BF16 tensor-core
    products with FP32 accumulation); the bias gradients stay exact."""
    rb = round_bf16 if bf16_operands else (lambda t: t)
    grads = [None] * len(params)
    p = len(params) - 1
    kind, h = cache[-1]
    grads[p] = _wgrad(h, dy, rb)
    g = conv3d_dgrad(rb(dy), params[p][0])
    p -= 1
    skip_grads = {}
    idx = len(cache) - 2
    for l in range(levels - 1):
        level = l  # decoder levels run 0 .. L-2 backwards from the output
        for _ in range(2):
            _, hin, a = cache[idx]
            g = g * (a > 0)
            grads[p] = _wgrad(hin, g, rb)
            g = conv3d_dgrad(rb(g), params[p][0])
            p -= 1
            idx -= 1
        _, nkept = cache[idx]
        skip_grads[level] = g[:nkept]
        g = up2_bwd(g[nkept:])
        idx -= 1
    for l in reversed(range(levels)):
        if l < levels - 1:
            _, shape = cache[idx]
            g = pool2_bwd(g) + skip_grads[l]
            idx -= 1
        for _ in range(2):
            _, hin, a = cache[idx]
            g = g * (a > 0)
            grads[p] = _wgrad(hin, g, rb)
            g = conv3d_dgrad(rb(g), params[p][0])
            p -= 1
            idx -= 1
    return grads
