"""FP64 NumPy oracle of the learned segment proposal and of the localisation
that uses it.

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this module. The CUDA library never does.

The learned proposal is not part of the paper. It replaces the segment
selection of Section III ("ROI Selection"), whose Eq. 5 decision metric stays
the fallback whenever the network is not confident. Its definition:

Network (3 layers of 3x3 convolutions, 32 channels, then a segment head)
  X0 = E / max(E)                       E: 32 x 32 coarse DAS energies (Eq. 3)
  A1 = q(relu(conv(X0; W1) + b1))       1 -> 32 channels
  A2 = q(relu(conv(A1; W2) + b2))       32 -> 32
  A3 = q(relu(conv(A2; W3) + b3))       32 -> 32
  F[s, c] = mean of A3[c] over segment s (16 segments: 8 x 8 map points each,
            s = 4 * (y // 8) + x // 8)
  z[s] = bh + sum_c wh[c] F[s, c]       16 segment scores
  p = softmax(z); confidence = max p; proposal = first argmax of z
Convolutions are zero padded, tap t = 3 (dy + 1) + (dx + 1), dy along the map
rows (grid axis 1), dx along the columns (grid axis 0):
  conv(X; W)[c, y, x] = sum_t sum_ci W[c, t, ci] X[ci, y + dy, x + dx].
q() rounds to bfloat16: conv weights are bfloat16, activations are stored in
bfloat16 and every sum accumulates in FP32 on the device (FP64 here), so the
oracle rounds at the same places and nowhere else.

Training: cross-entropy of softmax(z) against a segment label, averaged over
the batch; backward as the chain rule of the above, with the gradient at each
pre-activation rounded to bfloat16 (G_l = q(dZ_l)) before it meets the
weights; Adam with bias correction on FP32 master parameters.

Parameter vector theta (FP32), in this order:
  W1[32][9], b1[32], W2[32][9][32], b2[32], W3[32][9][32], b3[32], wh[32], bh[1]
"""
from __future__ import annotations

import numpy as np

MAP = 32            # coarse map side
CH = 32             # channels
TAPS = 9
SEG = 4             # segments per axis
SEG_SIDE = MAP // SEG
N_SEG = SEG * SEG

SIZES = [("W1", (CH, TAPS)), ("b1", (CH,)), ("W2", (CH, TAPS, CH)), ("b2", (CH,)),
         ("W3", (CH, TAPS, CH)), ("b3", (CH,)), ("wh", (CH,)), ("bh", (1,))]
N_PARAMS = int(sum(np.prod(s) for _, s in SIZES))


def unpack(theta: np.ndarray) -> dict:
    """Split the flat parameter vector into named FP64 arrays."""
    theta = np.asarray(theta, dtype=np.float64).ravel()
    if theta.size != N_PARAMS:
        raise ValueError(f"expected {N_PARAMS} parameters, got {theta.size}")
    out, off = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[off:off + n].reshape(shape).copy()
        off += n
    return out


def pack(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel()
                           for name, _ in SIZES])


def init_params(seed: int) -> np.ndarray:
    """He-normal conv weights, zero biases, small head (FP32 values)."""
    rng = np.random.Generator(np.random.Philox(seed))
    p = {
        "W1": rng.normal(0.0, np.sqrt(2.0 / TAPS), (CH, TAPS)),
        "b1": np.zeros(CH),
        "W2": rng.normal(0.0, np.sqrt(2.0 / (TAPS * CH)), (CH, TAPS, CH)),
        "b2": np.zeros(CH),
        "W3": rng.normal(0.0, np.sqrt(2.0 / (TAPS * CH)), (CH, TAPS, CH)),
        "b3": np.zeros(CH),
        "wh": rng.normal(0.0, np.sqrt(1.0 / CH), (CH,)),
        "bh": np.zeros(1),
    }
    return pack(p).astype(np.float32)


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via the FP32 value; returns FP64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def _ident(x):
    return np.asarray(x, dtype=np.float64)


def tap_offsets():
    """(dy, dx) of tap t = 3 (dy + 1) + (dx + 1)."""
    return [(t // 3 - 1, t % 3 - 1) for t in range(TAPS)]


def shifted(X: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """S[..., y, x] = X[..., y + dy, x + dx], zero outside the map."""
    S = np.zeros_like(X)
    H, W = X.shape[-2:]
    ys, yd = (slice(dy, H), slice(0, H - dy)) if dy >= 0 else (slice(0, H + dy), slice(-dy, H))
    xs, xd = (slice(dx, W), slice(0, W - dx)) if dx >= 0 else (slice(0, W + dx), slice(-dx, W))
    S[..., yd, xd] = X[..., ys, xs]
    return S


def conv(X: np.ndarray, W: np.ndarray) -> np.ndarray:
    """conv(X; W)[b, c, y, x] = sum_t sum_ci W[c, t, ci] X[b, ci, y + dy, x + dx].
    X: [B, Cin, H, W]; W: [Cout, 9, Cin]."""
    B, Cin, H, Wd = X.shape
    Z = np.zeros((B, W.shape[0], H, Wd))
    for t, (dy, dx) in enumerate(tap_offsets()):
        Z += np.einsum("oc,bcyx->boyx", W[:, t, :], shifted(X, dy, dx))
    return Z


def conv_input_grad(G: np.ndarray, W: np.ndarray) -> np.ndarray:
    """d/dX of sum(G * conv(X; W)): sum over taps of the weights applied to G
    shifted back by the tap offset."""
    B, Cout, H, Wd = G.shape
    D = np.zeros((B, W.shape[2], H, Wd))
    for t, (dy, dx) in enumerate(tap_offsets()):
        D += np.einsum("oc,boyx->bcyx", W[:, t, :], shifted(G, -dy, -dx))
    return D


def conv_weight_grad(G: np.ndarray, X: np.ndarray) -> np.ndarray:
    """d/dW of sum(G * conv(X; W)), summed over the batch: [Cout, 9, Cin]."""
    out = np.zeros((G.shape[1], TAPS, X.shape[1]))
    for t, (dy, dx) in enumerate(tap_offsets()):
        out[:, t, :] = np.einsum("boyx,bcyx->oc", G, shifted(X, dy, dx))
    return out


def normalise(E: np.ndarray) -> np.ndarray:
    """X0 = E / max(E) per map (all-zero maps stay zero). E: [B, 32, 32]."""
    E = np.asarray(E, dtype=np.float64)
    m = E.reshape(E.shape[0], -1).max(axis=1)
    scale = np.where(m > 0, 1.0 / np.where(m > 0, m, 1.0), 0.0)
    return E * scale[:, None, None]


def segment_pool(A: np.ndarray) -> np.ndarray:
    """F[b, s, c] = mean of A[b, c] over segment s. A: [B, C, 32, 32]."""
    B, C = A.shape[:2]
    blocks = A.reshape(B, C, SEG, SEG_SIDE, SEG, SEG_SIDE)
    return blocks.mean(axis=(3, 5)).transpose(0, 2, 3, 1).reshape(B, N_SEG, C)


def forward(theta, maps, quantise: bool = True) -> dict:
    """Scores and every intermediate. maps: [B, 32, 32] raw coarse energies."""
    q = bf16 if quantise else _ident
    P = unpack(theta)
    W1 = q(P["W1"])[:, :, None]                 # [32, 9, 1]
    W2, W3 = q(P["W2"]), q(P["W3"])
    X0 = normalise(maps)[:, None]               # [B, 1, 32, 32]
    A1 = q(np.maximum(conv(X0, W1) + P["b1"][None, :, None, None], 0.0))
    A2 = q(np.maximum(conv(A1, W2) + P["b2"][None, :, None, None], 0.0))
    A3 = q(np.maximum(conv(A2, W3) + P["b3"][None, :, None, None], 0.0))
    F = segment_pool(A3)                        # [B, 16, 32]
    z = F @ P["wh"] + P["bh"][0]                # [B, 16]
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    p = e / e.sum(axis=1, keepdims=True)
    return {"X0": X0, "A1": A1, "A2": A2, "A3": A3, "F": F, "z": z, "p": p,
            "W1": W1, "W2": W2, "W3": W3, "P": P}


def proposal(z: np.ndarray, p: np.ndarray, threshold: float):
    """(segment, confident) per map: the first argmax of z, and max p >= threshold."""
    seg = np.argmax(z, axis=1)
    conf = p.max(axis=1)
    return seg, conf >= threshold


def head_grad(dz: np.ndarray, F: np.ndarray):
    """Gradients of the head z[s] = bh + sum_c wh[c] F[s, c] for score
    gradients dz [B, 16] and segment means F [B, 16, 32]: (dwh [32], dbh [1])."""
    return np.einsum("bs,bsc->c", dz, F), np.array([dz.sum()])


def g3_from_dz(dz: np.ndarray, A3: np.ndarray, wh: np.ndarray, quantise: bool = True):
    """G3 = q(dA3 * [A3 > 0]): the gradient at layer 3's pre-activation, where
    dA3[c, y, x] = dz[segment of (y, x)] wh[c] / 64 (the segment mean's share)."""
    q = bf16 if quantise else _ident
    B = dz.shape[0]
    dF = dz[:, :, None] * wh[None, None, :]                 # [B, 16, 32]
    dA3 = np.repeat(np.repeat(
        dF.reshape(B, SEG, SEG, CH).transpose(0, 3, 1, 2), SEG_SIDE, axis=2),
        SEG_SIDE, axis=3) / (SEG_SIDE * SEG_SIDE)
    return q(dA3 * (A3 > 0))


def layer_grad(G: np.ndarray, A_in: np.ndarray):
    """Weight and bias gradients of conv(A_in; W) + b for its pre-activation
    gradient G: (dW [Cout, 9, Cin], db [Cout]), summed over the batch."""
    return conv_weight_grad(G, A_in), G.sum(axis=(0, 2, 3))


def input_grad(G: np.ndarray, W: np.ndarray, A_in: np.ndarray, quantise: bool = True):
    """The previous layer's pre-activation gradient q(conv^T(G; W) * [A_in > 0])."""
    q = bf16 if quantise else _ident
    return q(conv_input_grad(G, W) * (A_in > 0))


def loss_and_grad(theta, maps, labels, quantise: bool = True):
    """Mean cross-entropy and its gradient with respect to theta (flat)."""
    f = forward(theta, maps, quantise)
    B = maps.shape[0]
    labels = np.asarray(labels, dtype=np.int64)
    p = f["p"]
    loss = -np.mean(np.log(p[np.arange(B), labels]))
    dz = p.copy()
    dz[np.arange(B), labels] -= 1.0
    dz /= B
    P = f["P"]
    g = {}
    g["wh"], g["bh"] = head_grad(dz, f["F"])
    G3 = g3_from_dz(dz, f["A3"], P["wh"], quantise)
    g["W3"], g["b3"] = layer_grad(G3, f["A2"])
    G2 = input_grad(G3, f["W3"], f["A2"], quantise)
    g["W2"], g["b2"] = layer_grad(G2, f["A1"])
    G1 = input_grad(G2, f["W2"], f["A1"], quantise)
    dW1, g["b1"] = layer_grad(G1, f["X0"])
    g["W1"] = dW1[:, :, 0]
    return loss, pack(g)


def adam_step(theta, m, v, grad, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update with bias correction (step counts from 1)."""
    theta = np.asarray(theta, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ----------------------------------------------------------- learned localisation
def segment_box(lo: int, side: int, s: int):
    """Index box [lo', lo' + side / 4) per axis (x, y) of segment s of a square
    region [lo, lo + side)^2 (s = 4 * row + column)."""
    sub = side // SEG
    return (lo[0] + (s % SEG) * sub, lo[1] + (s // SEG) * sub), sub


def map_lattice(lo, side: int):
    """Lattice of the 32 x 32 coarse map of the square region [lo, lo + side)^2:
    point k at lo + o + step * k, step = side / 32, o = (step - 1) // 2."""
    step = side // MAP
    o = (step - 1) // 2
    return [lo[0] + o, lo[1] + o, 0], [step, step, 1], [MAP, MAP, 1]


def learned_localize(traces, antennas, grid: dict, v, fs, window, theta, threshold: float,
                     beamformer, rule, levels: int = 2, frame_num: int = 1,
                     frame_den: int = 4, localize=None, image=None) -> dict:
    """Localisation with the learned proposal (2-D square grids, side % 128 == 0).

    Each level images a 32 x 32 DAS map of the current square region, runs the
    network, and descends into the proposed segment (a quarter of the side per
    axis) when the confidence reaches the threshold. After the last level the
    segment is framed by ceil(frame_num / frame_den * side) points per side
    (Section III, sliding framing), imaged at full resolution with the
    requested beamformer and its first argmax taken. A level below the
    threshold hands the whole scan to the plain framework (Eq. 5 metric).
    `localize` / `image` are the oracle's plain-framework and imaging calls."""
    n = grid["n"][0]
    if grid["dim"] != 2 or grid["n"][1] != n or n % (MAP * SEG) != 0:
        raise ValueError("learned proposal needs a square 2-D grid with side % 128 == 0")
    lo, side = (0, 0), n
    segs, confs = [], []
    for _ in range(levels):
        l0, st, ct = map_lattice(lo, side)
        E = image(traces, antennas, grid, v, fs, window, 0, lo=l0, step=st, cnt=ct)[0]
        f = forward(theta, E[None])
        seg, ok = proposal(f["z"], f["p"], threshold)
        segs.append(int(seg[0]))
        confs.append(float(f["p"].max()))
        if not ok[0]:
            r = localize(traces, antennas, grid, v, fs, window, beamformer, rule)
            return {"fallback": True, "loc_idx": r["loc_idx"][:2], "segments": segs,
                    "confidence": confs, "framework": r}
        lo, side = segment_box(lo, side, int(seg[0]))
    fr = -(-frame_num * side // frame_den)
    blo = [max(lo[a] - fr, 0) for a in range(2)]
    bhi = [min(lo[a] + side + fr, n) for a in range(2)]
    cnt = [bhi[0] - blo[0], bhi[1] - blo[1], 1]
    img = image(traces, antennas, grid, v, fs, window, beamformer,
                lo=[blo[0], blo[1], 0], step=[1, 1, 1], cnt=cnt)[0]
    k = int(np.argmax(img))          # row-major [y][x]: the lowest linear index on ties
    y, x = divmod(k, cnt[0])
    return {"fallback": False, "loc_idx": [blo[0] + x, blo[1] + y], "segments": segs,
            "confidence": confs, "box_lo": blo, "box_hi": bhi, "peak": float(img.max())}
