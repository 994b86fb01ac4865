"""The element-wise network comparison (oracle/cnn_check.py) itself, on the CPU:
a record made by the oracle passes with every element exact, and a record
with a plausible kernel mistake planted in it fails at the step that made it."""
import numpy as np
import pytest

from oracle import cnn, cnn_check


def _case(seed=3, B=3):
    rng = np.random.Generator(np.random.Philox(seed))
    theta = cnn.init_params(seed).astype(np.float64)
    P = cnn.unpack(theta)
    for name in ("b1", "b2", "b3"):
        P[name] = rng.uniform(-0.05, 0.05, 32)
    P["wh"] *= 4.0
    theta = cnn.pack(P).astype(np.float32)
    maps = rng.gamma(2.0, 0.05, (B, 32, 32))
    maps[0, 9, 20] += 3.0
    maps = maps.astype(np.float32)
    labels = np.array([5, 0, 12][:B])
    return theta, maps, labels


def _records(theta, maps, labels):
    """Forward and after-gradient records as the kernels would write them, made
    by the oracle's own steps."""
    f = cnn.forward(theta, maps)
    B = maps.shape[0]
    fwd = {"X0": f["X0"][:, 0], "A1": f["A1"], "A2": f["A2"], "A3": f["A3"], "F": f["F"]}
    dz = f["p"].copy()
    dz[np.arange(B), labels] -= 1.0
    dz /= B
    dz = dz.astype(np.float32).astype(np.float64)
    G3 = cnn.g3_from_dz(dz, f["A3"], f["P"]["wh"])
    G2 = cnn.input_grad(G3, f["W3"], f["A2"])
    G1 = cnn.input_grad(G2, f["W2"], f["A1"])
    bwd = dict(fwd, A3=G2, A2=G1, dz=dz)
    fwd["dz"] = dz
    g = {}
    g["wh"], g["bh"] = cnn.head_grad(dz, f["F"])
    g["W3"], g["b3"] = cnn.layer_grad(G3, f["A2"])
    g["W2"], g["b2"] = cnn.layer_grad(G2, f["A1"])
    dW1, g["b1"] = cnn.layer_grad(G1, f["X0"])
    g["W1"] = dW1[:, :, 0]
    loss = -np.mean(np.log(f["p"][np.arange(B), labels]))
    return f, fwd, bwd, cnn.pack(g), loss


def test_oracle_made_records_pass_exactly():
    theta, maps, labels = _case()
    f, fwd, bwd, grad, loss = _records(theta, maps, labels)
    out = cnn_check.check_forward(theta, maps, fwd, f["z"])
    for step in ("A1", "A2", "A3", "F", "z"):
        assert out[step]["exact"] == out[step]["elements"], step
    out = cnn_check.check_backward(theta, labels, fwd, bwd, f["z"], grad, loss)
    for step in ("G2", "G1", "W3", "W2", "W1", "wh"):
        assert out[step]["exact"] == out[step]["elements"], step


def test_one_activation_off_by_two_bf16_steps_fails_at_its_layer():
    theta, maps, labels = _case()
    f, fwd, _, _, _ = _records(theta, maps, labels)
    bad = dict(fwd, A2=fwd["A2"].copy())
    c, y, x = np.argwhere(bad["A2"][1] > 0.1)[0]
    bad["A2"][1, c, y, x] += 2 * cnn_check.ulp_bf16(bad["A2"][1, c, y, x])
    with pytest.raises(AssertionError, match="A2"):
        cnn_check.check_forward(theta, maps, bad, f["z"])


def test_a_transposed_tap_fails():
    # a kernel reading the weights of tap (dy, dx) for tap (dx, dy)
    theta, maps, labels = _case()
    P = cnn.unpack(theta)
    perm = [3 * (t % 3) + t // 3 for t in range(9)]
    P["W3"] = P["W3"][:, perm, :]
    wrong = cnn.forward(cnn.pack(P), maps)
    f, fwd, _, _, _ = _records(theta, maps, labels)
    bad = dict(fwd, A3=wrong["A3"])
    with pytest.raises(AssertionError, match="A3"):
        cnn_check.check_forward(theta, maps, bad, f["z"])


def test_a_gradient_missing_one_map_border_fails():
    # a weight gradient that drops the contributions of one border row
    theta, maps, labels = _case()
    f, fwd, bwd, grad, loss = _records(theta, maps, labels)
    G3 = cnn.g3_from_dz(bwd["dz"], f["A3"], f["P"]["wh"])
    G3b = G3.copy()
    G3b[:, :, 31, :] = 0.0
    dW3, _ = cnn.layer_grad(G3b, f["A2"])
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in cnn.SIZES])
    k = [n for n, _ in cnn.SIZES].index("W3")
    bad = grad.copy()
    bad[offs[k]:offs[k + 1]] = dW3.ravel()
    if np.array_equal(bad, grad):
        pytest.skip("the border row carries no gradient for these maps")
    with pytest.raises(AssertionError, match="W3"):
        cnn_check.check_backward(theta, labels, fwd, bwd, f["z"], bad, loss)


def test_bf16_spacing():
    assert cnn_check.ulp_bf16(np.array([1.0]))[0] == 2.0 ** -7
    assert cnn_check.ulp_bf16(np.array([1.99]))[0] == 2.0 ** -7
    assert cnn_check.ulp_bf16(np.array([2.0]))[0] == 2.0 ** -6
    assert cnn_check.ulp_bf16(np.array([0.0]))[0] == 0.0
    # consecutive BF16 values differ by exactly that spacing
    x = cnn.bf16(np.array([1.3]))[0]
    bits = np.array([x], np.float32).view(np.uint32)[0] + (1 << 16)
    nxt = np.array([bits], np.uint32).view(np.float32)[0]
    assert nxt - x == cnn_check.ulp_bf16(np.array([x]))[0]


def test_record_decoder_follows_the_documented_layout():
    """paper_1709_02549_gb300.cnn_record_arrays against bytes placed by hand at
    the offsets the header documents (X0 float at 4u, channel c of a BF16 map
    at base + (c / 8) 19616 + 16 u + 2 (c % 8), u = 34 + 33 y + x; F at 240512,
    dz at 242560)."""
    import paper_1709_02549_gb300 as uwb
    B = 2
    raw = np.zeros(B * uwb.CNN_RECORD_BYTES, np.uint8)
    rec = raw.reshape(B, uwb.CNN_RECORD_BYTES)

    def put_f32(b, off, v):
        rec[b, off:off + 4] = np.frombuffer(np.float32(v).tobytes(), np.uint8)

    def put_bf16(b, off, v):
        bits = np.array([v], np.float32).view(np.uint32)[0] >> 16
        rec[b, off] = bits & 0xFF
        rec[b, off + 1] = bits >> 8

    u = 34 + 33 * 7 + 19                      # y = 7, x = 19
    put_f32(1, 4 * u, 0.75)
    for name, base, c, v in (("A1", 5120, 13, 1.5), ("A2", 83584, 0, -2.0),
                             ("A3", 162048, 31, 0.125)):
        put_bf16(1, base + (c // 8) * 19616 + 16 * u + 2 * (c % 8), v)
    put_f32(0, 240512 + 4 * (5 * 32 + 9), 3.25)
    put_f32(0, 242560 + 4 * 15, -0.5)
    arr = uwb.cnn_record_arrays(raw, B)
    assert arr["X0"][1, 7, 19] == 0.75 and np.count_nonzero(arr["X0"]) == 1
    assert arr["A1"][1, 13, 7, 19] == 1.5 and np.count_nonzero(arr["A1"]) == 1
    assert arr["A2"][1, 0, 7, 19] == -2.0 and np.count_nonzero(arr["A2"]) == 1
    assert arr["A3"][1, 31, 7, 19] == 0.125 and np.count_nonzero(arr["A3"]) == 1
    assert arr["F"][0, 5, 9] == 3.25 and np.count_nonzero(arr["F"]) == 1
    assert arr["dz"][0, 15] == -0.5 and np.count_nonzero(arr["dz"]) == 1
