"""Pins for the learned-guess reference: gradients against central finite differences, the
Adam update against its closed form for one step, and the SH projection round trip."""
import numpy as np

import synth
from oracle import mlp
from oracle import timestep as ts


def test_gradients_match_finite_differences():
    rng = np.random.Generator(np.random.PCG64(1))
    params = mlp.init_params((7, 6, 6, 6, 5), seed=3)
    F = rng.standard_normal((9, 7))
    T = rng.standard_normal((9, 5))
    L, grads = mlp.loss_and_grads(params, F, T)
    h = 1e-6
    for i in range(len(params)):
        for j in range(2):
            P = params[i][j]
            idx = [tuple(rng.integers(0, s) for s in P.shape) for _ in range(4)]
            for k in idx:
                old = P[k]
                P[k] = old + h
                Lp, _ = mlp.loss_and_grads(params, F, T)
                P[k] = old - h
                Lm, _ = mlp.loss_and_grads(params, F, T)
                P[k] = old
                fd = (Lp - Lm) / (2 * h)
                assert abs(fd - grads[i][j][k]) < 1e-6 * max(1.0, abs(fd))


def test_adam_first_step_moves_by_lr_times_sign():
    # with zero moments, the bias-corrected first step is -lr * g / (|g| + eps) ~ -lr sign(g)
    params = [[np.array([[1.0, -2.0]]), np.array([0.5])]]
    grads = [[np.array([[0.3, -0.7]]), np.array([2.0])]]
    st = {}
    mlp.adam_step(params, grads, st, lr=0.01)
    assert np.allclose(params[0][0], [[0.99, -1.99]], atol=1e-7)
    assert np.allclose(params[0][1], [0.49], atol=1e-7)


def test_training_reduces_loss_on_a_learnable_map():
    rng = np.random.Generator(np.random.PCG64(2))
    A = rng.standard_normal((4, 6)) * 0.5
    F = rng.standard_normal((64, 6))
    T = F @ A.T
    params = mlp.init_params((6, 32, 32, 32, 4), seed=4)
    st = {}
    L0, _ = mlp.loss_and_grads(params, F, T)
    for _ in range(300):
        L, g = mlp.loss_and_grads(params, F, T)
        mlp.adam_step(params, g, st, lr=3e-3)
    assert L < 0.05 * L0


def test_sh_projection_round_trip():
    v, _ = synth.icosphere(3)
    G, Gp = ts.filter_factors(v, 11)  # l <= 10: 121 coefficients
    c = np.random.Generator(np.random.PCG64(5)).standard_normal(121)
    x = G @ c
    vert_off = np.array([0, 642, 1284])
    X = np.concatenate([x, 2 * x])
    C = mlp.sh_coefficients([Gp], X, vert_off, [0, 0])
    assert np.allclose(C[0], c, atol=1e-9) and np.allclose(C[1], 2 * c, atol=1e-9)
    assert np.allclose(mlp.sh_synthesis([G], C, vert_off, [0, 0]), X, atol=1e-9)


def test_bf16_rounding_is_round_to_nearest_even():
    # values with at most 8 significant bits are exact; halfway cases go to the even neighbour
    exact = np.array([1.0, -1.5, 0.75, 2.0 ** -20, 3.0 * 2.0 ** 7, 1.0 + 2.0 ** -7])
    assert np.array_equal(mlp.bf16(exact), exact)
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0                      # tie -> even (1.0000000)
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6      # tie -> even (1.0000010)
    assert mlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7  # above the tie -> up
    assert mlp.bf16(-(1.0 + 3 * 2.0 ** -8)) == -(1.0 + 2.0 ** -6)
    x = np.random.Generator(np.random.PCG64(3)).standard_normal(100000) * 10.0 ** np.linspace(-6, 6, 100000)
    r = mlp.bf16(x)
    rel = np.abs(r - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -8 * (1 + 1e-6)  # half a unit in the 8th significant bit
    assert np.array_equal(mlp.bf16(r), r)


def test_bf16_network_reduces_to_the_plain_one_without_rounding_and_costs_a_few_percent():
    rng = np.random.Generator(np.random.PCG64(8))
    params = mlp.init_params((48, 64, 64, 64, 16), seed=7)
    F = rng.standard_normal((200, 48))
    T = rng.standard_normal((200, 16)) * 0.3
    ident = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731
    Y, _ = mlp.forward(params, F)
    Yi, _ = mlp.forward_bf16(params, F, rnd=ident)
    assert np.allclose(Yi, Y, rtol=0, atol=1e-13)
    L, g = mlp.loss_and_grads(params, F, T)
    Li, gi = mlp.loss_and_grads_bf16(params, F, T, rnd=ident)
    assert abs(Li - L) < 1e-13 * L
    for a, b in zip(gi, g):
        assert np.allclose(a[0], b[0], atol=1e-13) and np.allclose(a[1], b[1], atol=1e-13)
    # the BF16 rounding itself: the measured error budget of a BF16-operand network against
    # FP64 (8 significant bits per operand, four layers): forward ~0.5-1e-2, loss ~1e-2,
    # per-layer weight gradients a few 1e-2
    Yb, _ = mlp.forward_bf16(params, F)
    Lb, gb = mlp.loss_and_grads_bf16(params, F, T)
    ef = np.linalg.norm(Yb - Y) / np.linalg.norm(Y)
    el = abs(Lb - L) / L
    eg = [np.linalg.norm(a[0] - b[0]) / np.linalg.norm(b[0]) for a, b in zip(gb, g)]
    print("BF16 vs FP64: forward %.3g, loss %.3g, weight gradients %s" % (ef, el, ["%.3g" % e for e in eg]))
    assert 1e-4 < ef < 3e-2 and el < 3e-2 and max(eg) < 1e-1
