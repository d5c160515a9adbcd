"""Precision of the tensor-core tiles of the learned closure, emulated on the
CPU against the FP64 oracle (no GPU).

The tiles evaluate the network with the BF16 weight values held as FP16
operands, FP16 normalised inputs, FP16 accumulators for the hidden layers
(rounded after every K = 16 instruction, the bias block included), the SiLU
as h + h tanh(h) on FP16 pairs (tanh and the fused multiply-add each rounded
once to FP16), and an FP32 output layer with hi/lo output weights.  This
test rounds the same way in NumPy and checks the result against the
oracle's forward pass with the forward gate of the GPU test (2e-2 relative
+ 1e-3 of the largest value), on the GPU test's network and inputs.  The
same arithmetic with the activations rounded to BF16 (8 significant bits
against 11) is measured beside it: 0.63 of the gate at its worst row, about
three times the FP16 tiles' error.
"""
import numpy as np

H, I = 64, 6


def _bf16(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _f16(a):
    return np.asarray(a, dtype=np.float64).astype(np.float16).astype(np.float64)


def _split(theta):
    off, out = 0, {}
    for name, n in (("w1", H * I), ("b1", H), ("w2", H * H), ("b2", H), ("w3", H * H), ("b3", H), ("w4", H),
                    ("b4", 1)):
        out[name] = theta[off:off + n].astype(np.float64)
        off += n
    return out


def _features(O, rng, n, nu=1e-3):
    G = rng.standard_normal((n, 3, 3)) * rng.uniform(0.1, 3.0, (n, 1, 1))
    delta = rng.uniform(0.005, 0.05, n)
    return np.stack([O.mlp_features(G[k], delta[k], nu) for k in range(n)]).astype(np.float32)


def _layer(a, W, b, act_round):
    """Hidden layer of the tiles: halved FP16 weights, FP16 accumulation per
    K = 16 block (then the bias block), SiLU on FP16 values."""
    acc = np.zeros((a.shape[0], W.shape[0]))
    for k0 in range(0, a.shape[1], 16):
        acc = _f16(acc + a[:, k0:k0 + 16] @ (0.5 * W[:, k0:k0 + 16]).T)
    h = _f16(acc + 0.5 * b)
    t = _f16(np.tanh(h))
    return act_round(h + h * t)


def _tiles_forward(theta, xn, scale, act_round=_f16):
    p = _split(theta)
    W1, W2, W3 = (_bf16(p[k]).reshape(H, -1) for k in ("w1", "w2", "w3"))
    a = _layer(_f16(xn), W1, p["b1"], act_round)
    a = _layer(a, W2, p["b2"], act_round)
    a = _layer(a, W3, p["b3"], act_round)
    z = a @ p["w4"] + p["b4"][0]
    return scale * np.log1p(np.exp(z))


def _oracle_forward(O, theta, xn, scale):
    t = theta.astype(np.float64).copy()
    p = _split(theta)
    off = 0
    for name, n in (("w1", H * I), ("b1", H), ("w2", H * H), ("b2", H), ("w3", H * H), ("b3", H)):
        if name in ("w1", "w2", "w3"):
            t[off:off + n] = _bf16(p[name])
        off += n
    mlp = O.MLPParams(t, np.zeros(6), np.ones(6), scale)
    return O.mlp_forward(mlp, xn)


def test_fp16_tiles_meet_the_forward_gate(oracle_lib):
    O = oracle_lib
    from paper_2005_05899_b300 import fea
    rng = np.random.default_rng(0)
    theta = (0.3 * rng.standard_normal(fea.MLP_NPARAM)).astype(np.float32)
    x = _features(O, rng, 3000)
    mean = x.mean(axis=0).astype(np.float32)
    std = (x.std(axis=0) + 1e-3).astype(np.float32)
    scale = 2e-4
    xn = _f16((x - mean) / std)
    ref = _oracle_forward(O, theta, xn, scale)
    tol = 2e-2 * np.abs(ref) + 1e-3 * np.abs(ref).max()
    got = _tiles_forward(theta, xn, scale)
    worst = np.max(np.abs(got - ref) / tol)
    assert worst < 0.5, worst
    # the same arithmetic with BF16 activations: within the gate here, but
    # with about three times the error at the worst row
    got_bf16 = _tiles_forward(theta, xn, scale, act_round=_bf16)
    worst_bf16 = np.max(np.abs(got_bf16 - ref) / tol)
    assert worst_bf16 > 2.0 * worst, (worst, worst_bf16)
