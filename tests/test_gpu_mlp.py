"""The learned initial guess on the device: forward pass and gradients of the BF16
tensor-core network against the FP64 CPU reference (oracle/mlp.py), and a short
record-train-use run showing what the trained network gains over the previous-step guess."""
import numpy as np
import pytest

import synth
from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bem():
    from paper_1905_01341_gb300 import bem

    return bem


def _unflatten(flat, dims):
    params, off = [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        W = flat[off:off + a * b].reshape(b, a)
        off += a * b
        bb = flat[off:off + b]
        off += b
        params.append([W.copy(), bb.copy()])
    return params


def _flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def small_system(nb=8, level=3, seed=6):
    rng = np.random.Generator(np.random.PCG64(seed))
    radii = np.exp(0.3 * rng.standard_normal(nb))
    box = max(4.0 * nb ** (1 / 3), 4.0 * radii.max())
    centres = synth._place_centres(radii, box, 0.5, rng)
    mesh = synth.cluster(level, radii, centres)
    phi = synth.cluster_potential(mesh, 4, 0.05, rng) - 1.0
    return mesh, phi


def make_stepper(mesh, phi, guess=0, **params):
    bem = _bem()
    ctx = bem.BemContext(**params)
    ctx.upload_mesh(mesh)
    bem.bem_step_init(ctx.ctx, phi, bem.bem_step_params_default(pa=0.5, pf=6, guess=guess))
    return ctx


def test_forward_and_gradients_match_reference():
    bem = _bem()
    mesh, phi = small_system(4)
    ctx = make_stepper(mesh, phi, mvp=bem.BEM_MVP_DIRECT, precision=bem.BEM_PREC_FP64)
    bem.bem_mlp_init(ctx.ctx, hidden=64, lmax=3, seed=7)
    info = bem.bem_mlp_info(ctx.ctx)
    dims = info["dims"]
    assert dims == [48, 64, 64, 64, 16]
    flat = np.zeros(info["num_params"])
    bem.bem_mlp_get_params(ctx.ctx, flat)
    params = _unflatten(flat, dims)
    rng = np.random.Generator(np.random.PCG64(8))
    B = 200  # two row tiles with a ragged tail
    F = rng.standard_normal((B, dims[0]))
    T = rng.standard_normal((B, dims[4])) * 0.3
    Y = np.zeros((B, dims[4]))
    bem.bem_mlp_forward(ctx.ctx, F, Y)
    # the reference takes the products' operands in BF16, as the network's arithmetic is
    # stated (BF16 weights, features, activations and back-propagated errors; FP32 sums on the
    # device, FP64 in the reference): the two agree to the sums' rounding
    Yref, _ = omlp.forward_bf16(params, F)
    ef = np.linalg.norm(Y - Yref) / np.linalg.norm(Yref)
    g = np.zeros(info["num_params"])
    loss = bem.bem_mlp_loss_grad(ctx.ctx, F, T, g)
    Lref, gref = omlp.loss_and_grads_bf16(params, F, T)
    el = abs(loss - Lref) / Lref
    gflat = _flatten(gref)
    eg = np.linalg.norm(g - gflat) / np.linalg.norm(gflat)
    # each layer's weight and bias gradient separately (a transposed operand in one product
    # would give an O(1) error here)
    gl = _unflatten(g, dims)
    ew = [np.linalg.norm(a[0] - b[0]) / np.linalg.norm(b[0]) for a, b in zip(gl, gref)]
    eb = [np.linalg.norm(a[1] - b[1]) / np.linalg.norm(b[1]) for a, b in zip(gl, gref)]
    # for the record: the same network without rounding (the BF16 rounding's own cost)
    Y64, _ = omlp.forward(params, F)
    _, g64 = omlp.loss_and_grads(params, F, T)
    print("vs BF16-operand reference: forward %.3g, loss %.3g, gradient %.3g, per-layer W %s, b %s; "
          "vs FP64 without rounding: forward %.3g, per-layer W %s" % (
              ef, el, eg, ["%.3g" % e for e in ew], ["%.3g" % e for e in eb],
              np.linalg.norm(Y - Y64) / np.linalg.norm(Y64),
              ["%.3g" % (np.linalg.norm(a[0] - b[0]) / np.linalg.norm(b[0])) for a, b in zip(gl, g64)]))
    tol = 1e-2  # relative L2, the contract for the BF16 network's forward pass, loss and gradients
    assert ef < tol and el < tol and eg < tol
    assert max(ew) < tol and max(eb) < tol
    ctx.close()


def test_trained_guess_reduces_gmres_iterations():
    """Record the solves of 40 steps (35 in the Adams-Bashforth phase), train, then step on
    with the learned guess while also solving from its base start, the previous step's q (the
    paper's start, guess = 0): the learned start has the smaller initial residual and needs fewer
    GMRES iterations in total. (Against the extrapolated start, guess = 2, the benchmark reports
    the comparison; there the extrapolation already leaves a residual near the solves' own
    accuracy and the learned correction gains little.)"""
    bem = _bem()
    mesh, phi = small_system(8)
    ctx = make_stepper(mesh, phi, mvp=bem.BEM_MVP_DIRECT, precision=bem.BEM_PREC_FP64, gmres_tol=1e-8)
    bem.bem_mlp_init(ctx.ctx, hidden=128, lmax=6, seed=1)
    bem.bem_mlp_set_mode(ctx.ctx, record=True)
    for _ in range(40):
        bem.bem_step(ctx.ctx)
    info = bem.bem_mlp_info(ctx.ctx)
    assert info["samples"] == 35 * 8
    loss0 = bem.bem_mlp_train(ctx.ctx, epochs=1, batch=64, lr=1e-3)
    loss = bem.bem_mlp_train(ctx.ctx, epochs=200, batch=64, lr=1e-3)
    assert loss < loss0
    bem.bem_mlp_set_mode(ctx.ctx, record=False, use_guess=True, compare=True)
    for _ in range(10):
        bem.bem_step(ctx.ctx)
    info = bem.bem_mlp_info(ctx.ctx)
    print("mlp compare:", info)
    assert info["compared_solves"] == 10
    assert info["res0_guess"] < info["res0_fallback"]
    assert info["iters_guess"] < info["iters_fallback"]
    ctx.close()
