"""Element-wise comparison of the network kernels' record against the FP64
oracle of oracle/cnn.py, one step at a time.

TEST INFRASTRUCTURE: only the test suite and ``__graft_entry__.smoke()`` use
this module. The CUDA library never does.

Each step of the network is recomputed by the oracle from the kernels' own
stored inputs of that step (the BF16 activations, the FP32 segment means and
score gradients of the record), so that an error is caught where it is made
and does not propagate. The bounds follow from where the kernels round:

* a sum of K terms accumulated in FP32, in any order, by any adder whose
  every step is off by at most one FP32 ulp of its result (round to nearest
  on the CUDA cores; the tensor cores' accumulation is also covered): its
  error is at most K * 2^-23 * sum |term|. Products of two BF16 values are
  exact in FP32, and the CUDA cores' multiply-adds round once;
* a value then rounded to BF16 (after the ReLU, which is 1-Lipschitz) moves
  by at most one BF16 ulp of its magnitude (8 significant bits):
  |q(a) - q(b)| <= |a - b| + ulp_bf16(max(|a|, |b|)).
"""
from __future__ import annotations

import numpy as np

from . import cnn

ULP32 = 2.0 ** -23


def ulp_bf16(v: np.ndarray) -> np.ndarray:
    """Spacing of BF16 values at magnitude v (0 where v is 0)."""
    v = np.abs(np.asarray(v, dtype=np.float64))
    out = np.zeros_like(v)
    nz = v > 0
    out[nz] = 2.0 ** (np.floor(np.log2(v[nz])) - 7)
    return out


def _close(name: str, got, ref, tol) -> dict:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    tol = np.broadcast_to(np.asarray(tol, dtype=np.float64), ref.shape)
    err = np.abs(got - ref)
    bad = err > tol
    if np.any(bad):
        k = int(np.flatnonzero(bad.ravel())[0])
        raise AssertionError(f"{name}: {int(bad.sum())} of {bad.size} elements outside the "
                             f"bound; first at flat index {k}: gpu {got.ravel()[k]!r}, oracle "
                             f"{ref.ravel()[k]!r}, bound {np.ravel(tol)[k]!r}")
    return {"elements": int(got.size), "exact": int(np.sum(err == 0)),
            "max_err_over_bound": float(np.max(np.where(tol > 0, err / np.where(tol > 0, tol, 1),
                                                        0.0))) if got.size else 0.0}


def check_layer(name: str, A_in, W, b, A_gpu) -> dict:
    """A_gpu (the kernels' BF16 output of one layer) against
    q(relu(conv(A_in; W) + b)) computed from the kernels' own input A_in."""
    pre = cnn.conv(A_in, W) + b[None, :, None, None]
    absum = cnn.conv(np.abs(A_in), np.abs(W)) + np.abs(b)[None, :, None, None]
    K = W.shape[1] * W.shape[2] + 1
    e = K * ULP32 * absum
    ref = cnn.bf16(np.maximum(pre, 0.0))
    return _close(name, A_gpu, ref, e + ulp_bf16(np.abs(ref) + e))


def check_forward(theta, maps, rec: dict, scores_gpu) -> dict:
    """Every step of the forward pass of the maps in `rec` (decoded record
    arrays, batch-first) against the oracle fed with the kernels' own inputs."""
    P = cnn.unpack(theta)
    W1 = cnn.bf16(P["W1"])[:, :, None]
    W2, W3 = cnn.bf16(P["W2"]), cnn.bf16(P["W3"])
    out = {}
    # X0 = E * (1 / max E): a rounded reciprocal and a rounded product
    x0 = cnn.normalise(maps)
    out["X0"] = _close("X0", rec["X0"], x0, 2.01 * ULP32 * np.abs(x0))
    out["A1"] = check_layer("A1", rec["X0"][:, None], W1, P["b1"], rec["A1"])
    out["A2"] = check_layer("A2", rec["A1"], W2, P["b2"], rec["A2"])
    out["A3"] = check_layer("A3", rec["A2"], W3, P["b3"], rec["A3"])
    # segment means: 64 BF16 values summed in FP32, times 1/64 (exact)
    F = cnn.segment_pool(rec["A3"])
    eF = 64 * ULP32 * cnn.segment_pool(np.abs(rec["A3"]))
    out["F"] = _close("F", rec["F"], F, eF)
    # scores from the kernels' segment means: bh + 32 multiply-adds
    z = rec["F"] @ P["wh"] + P["bh"][0]
    ez = 33 * ULP32 * (np.abs(rec["F"]) @ np.abs(P["wh"]) + abs(P["bh"][0]))
    out["z"] = _close("z", scores_gpu, z, ez)
    return out


def check_backward(theta, labels, fwd: dict, bwd: dict, scores_gpu, grad_gpu, loss_gpu) -> dict:
    """Every step of the backward pass against the oracle fed with the kernels'
    own stored values. fwd: the forward record (A2, A3 intact); bwd: the
    record after the gradient call (A2 slot = G1, A3 slot = G2, dz written)."""
    P = cnn.unpack(theta)
    W2, W3 = cnn.bf16(P["W2"]), cnn.bf16(P["W3"])
    z = np.asarray(scores_gpu, dtype=np.float64)
    B = z.shape[0]
    lab = np.asarray(labels, dtype=np.int64)
    out = {}
    # the forward parts the backward pass reads are the forward record's
    for key in ("X0", "A1", "F"):
        if not np.array_equal(fwd[key], bwd[key]):
            raise AssertionError(f"{key} differs between the forward and gradient records")
    # dz = (softmax(z) - onehot) / B from the kernels' scores: expf within 2
    # ulp, a 16-term sum and a division
    zr = z - z.max(axis=1, keepdims=True)
    p = np.exp(zr)
    s = p.sum(axis=1, keepdims=True)
    p = p / s
    onehot = np.zeros_like(p)
    onehot[np.arange(B), lab] = 1.0
    dz = (p - onehot) / B
    rel_p = (2 * 2 + 16 + 2) * ULP32 + ULP32 * np.abs(zr).max(axis=1, keepdims=True)
    out["dz"] = _close("dz", bwd["dz"], dz, (rel_p * p + ULP32 * np.abs(p - onehot)) / B * 1.01)
    # loss from the kernels' scores: log of the sum and the label's score
    lb = np.log(s[:, 0]) - zr[np.arange(B), lab]
    el = (rel_p[:, 0] + 2 * ULP32 * (np.abs(np.log(s[:, 0])) + np.abs(zr[np.arange(B), lab]))
          + (B + 1) * ULP32 * np.abs(lb))
    out["loss"] = _close("loss", [float(loss_gpu)], [lb.mean()], [el.sum() / B])
    dzg = bwd["dz"]
    # G3 from the kernels' dz: a product of two FP32 values, rounded to FP32
    # and then to BF16, as the oracle rounds it; no tolerance needed after it
    G3 = cnn.g3_from_dz(dzg, fwd["A3"], P["wh"])
    G2, G1 = bwd["A3"], bwd["A2"]

    def check_input_grad(name, G, W, A_in, got):
        ref = cnn.input_grad(G, W, A_in)
        e = W.shape[0] * W.shape[1] * ULP32 * np.abs(cnn.conv_input_grad(np.abs(G), np.abs(W)))
        return _close(name, got, ref, e + ulp_bf16(np.abs(ref) + e))

    out["G2"] = check_input_grad("G2", G3, W3, fwd["A2"], G2)
    out["G1"] = check_input_grad("G1", G2, W2, fwd["A1"], G1)
    # parameter gradients: sums over the batch and the 1024 positions, with
    # one more addition per map and one atomic addition per CTA
    offs = np.cumsum([0] + [int(np.prod(sh)) for _, sh in cnn.SIZES])
    got = {name: np.asarray(grad_gpu[offs[k]:offs[k + 1]], dtype=np.float64).reshape(sh)
           for k, (name, sh) in enumerate(cnn.SIZES)}
    n = B * (cnn.MAP * cnn.MAP + 2)
    X0 = fwd["X0"][:, None]
    for layer, G, A_in in ((3, G3, fwd["A2"]), (2, G2, fwd["A1"]), (1, G1, X0)):
        dW, db = cnn.layer_grad(G, A_in)
        adW, adb = cnn.layer_grad(np.abs(G), np.abs(A_in))
        if layer == 1:
            dW, adW = dW[:, :, 0], adW[:, :, 0]
        out[f"W{layer}"] = _close(f"W{layer}", got[f"W{layer}"], dW, n * ULP32 * adW)
        out[f"b{layer}"] = _close(f"b{layer}", got[f"b{layer}"], db, n * ULP32 * adb)
    dwh, dbh = cnn.head_grad(dzg, fwd["F"])
    adwh, adbh = cnn.head_grad(np.abs(dzg), np.abs(fwd["F"]))
    m = B * (cnn.N_SEG + 2)
    out["wh"] = _close("wh", got["wh"], dwh, m * ULP32 * adwh)
    out["bh"] = _close("bh", got["bh"], dbh, m * ULP32 * adbh)
    return out
