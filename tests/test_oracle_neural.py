"""Pins of the learned-form oracle (CPU only): codecs against torch/numpy casts, features
against an independent bilinear, MLP forward/backward against torch float64 autograd and
central finite differences, Adam against its closed-form first step."""
import math

import numpy as np
import pytest
import torch

import oracle
import stf_synth as synth


def test_codecs_match_library_casts():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 1, 3000), rng.normal(0, 1e-3, 500), rng.normal(0, 100, 500),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0, 3e-8]]).astype(np.float32)
    bf = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.round_bf16(x), bf)
    np.testing.assert_array_equal(oracle.round_fp16(x), x.astype(np.float16).astype(np.float64))
    inr = x[np.abs(x) <= 448.0]
    f8 = torch.from_numpy(inr).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.round_e4m3(inr), f8)
    # E4M3 saturates at +-448 (no infinities), and decodes its 254 finite codes exactly
    assert oracle.round_e4m3(1e6) == 448.0 and oracle.round_e4m3(-500.0) == -448.0
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = oracle.e4m3_value(codes)
    fin = ~np.isnan(ref)
    np.testing.assert_array_equal(got[fin], ref[fin])
    assert np.all(np.isnan(got[~fin]))


def _small_net(seed=3, tex_res=32, grids=(16, 8, 4, 2)):
    lat, mlp = synth.ntc_init(grids, seed)
    return lat, mlp, tex_res


def test_features_match_float64_bilinear():
    lat, mlp, R0 = _small_net()
    nt = oracle.NeuralTexture(R0, lat, np.zeros(6792), "fp32")
    ix, iy = np.meshgrid(np.arange(R0), np.arange(R0))
    ix, iy = ix.ravel(), iy.ravel()
    f = oracle.ntc_features(nt, ix, iy)
    for g, G in enumerate(lat):
        R = G.shape[0]
        px = (ix + 0.5) * R / R0 - 0.5
        py = (iy + 0.5) * R / R0 - 0.5
        x0, y0 = np.floor(px).astype(int), np.floor(py).astype(int)
        tx, ty = px - x0, py - y0
        Gd = G.astype(np.float64)
        v = ((1 - tx) * (1 - ty))[:, None] * Gd[y0 % R, x0 % R] + (tx * (1 - ty))[:, None] * Gd[y0 % R, (x0 + 1) % R] \
            + ((1 - tx) * ty)[:, None] * Gd[(y0 + 1) % R, x0 % R] + (tx * ty)[:, None] * Gd[(y0 + 1) % R, (x0 + 1) % R]
        np.testing.assert_allclose(f[:, 8 * g:8 * g + 8], v, atol=3e-8)


def _torch_forward(L, M, ix, iy, R0):
    """Independent float64 restatement of the decode: bilinear features of the grids L (wrap,
    at texel centres), MLP M (no BF16 rounding)."""
    W1, b1 = M[:2048].view(64, 32), M[2048:2112]
    W2, b2 = M[2112:6208].view(64, 64), M[6208:6272]
    W3, b3 = M[6272:6784].view(8, 64), M[6784:6792]
    feats = []
    ixt, iyt = torch.tensor(ix, dtype=torch.float64), torch.tensor(iy, dtype=torch.float64)
    for G in L:
        R = G.shape[0]
        px = (ixt + 0.5) * R / R0 - 0.5
        py = (iyt + 0.5) * R / R0 - 0.5
        x0, y0 = torch.floor(px), torch.floor(py)
        tx, ty = (px - x0)[:, None], (py - y0)[:, None]
        x0, y0 = x0.long() % R, y0.long() % R
        x1, y1 = (x0 + 1) % R, (y0 + 1) % R
        feats.append((1 - tx) * (1 - ty) * G[y0, x0] + tx * (1 - ty) * G[y0, x1]
                     + (1 - tx) * ty * G[y1, x0] + tx * ty * G[y1, x1])
    x = torch.cat(feats, 1)
    h1 = torch.relu(x @ W1.T + b1)
    h2 = torch.relu(h1 @ W2.T + b2)
    return h2 @ W3.T + b3


def _torch_loss(lat, mlp, targets, ix, iy, R0):
    """Independent float64 restatement: bilinear features, MLP, MSE (no BF16 rounding)."""
    L = [torch.tensor(g, dtype=torch.float64, requires_grad=True) for g in lat]
    M = torch.tensor(mlp, dtype=torch.float64, requires_grad=True)
    y = _torch_forward(L, M, ix, iy, R0)
    t = torch.tensor(targets[iy, ix], dtype=torch.float64) / 255.0
    loss = ((y - t) ** 2).mean()
    loss.backward()
    return float(loss.detach()), M.grad.numpy(), np.concatenate([g.grad.numpy().ravel() for g in L])


def test_exact_decode_matches_torch_float64():
    # the exact FP64 decode (the reference of the inference forms' decode error) against the
    # independent torch float64 forward, on every texel of a small network
    lat, mlp, R0 = _small_net()
    mlp[2048:2112] = 0.05
    ix, iy = np.meshgrid(np.arange(R0), np.arange(R0))
    ix, iy = ix.ravel(), iy.ravel()
    y = oracle.ntc_decode_exact(R0, lat, mlp, ix, iy)
    with torch.no_grad():
        t = _torch_forward([torch.tensor(g, dtype=torch.float64) for g in lat],
                           torch.tensor(np.asarray(mlp, np.float32), dtype=torch.float64), ix, iy, R0).numpy()
    np.testing.assert_allclose(y, t, rtol=1e-12, atol=1e-13)
    # the FP16 inference form (BF16 weights and activations, FP16 latents) differs from it by
    # the quantisation, a few 1e-3 here, not by an error of the decode itself
    yq, _ = oracle.ntc_decode(oracle.NeuralTexture.inference_form(R0, lat, mlp, "fp16"), ix, iy)
    assert 1e-5 < np.sqrt(np.mean((yq - y) ** 2)) < 2e-2


def test_loss_and_gradients_match_torch_autograd():
    lat, mlp, R0 = _small_net()
    mlp[2048:2112] = 0.05                       # positive biases keep most ReLUs active
    m = synth.material_rgba8(R0, 7, octaves=3, base=2, mips=False)
    targets = synth.ntc_targets(m, 9)
    rng = np.random.default_rng(4)
    ix, iy = rng.integers(0, R0, 300), rng.integers(0, R0, 300)
    loss, gm, gl = oracle.ntc_loss_grad(R0, lat, mlp, targets, ix, iy, round_bf16=False)
    tl, tgm, tgl = _torch_loss(lat, mlp, targets, ix, iy, R0)
    assert abs(loss - tl) <= 1e-6 * tl
    np.testing.assert_allclose(gm, tgm, rtol=1e-5, atol=1e-9 * np.abs(tgm).max())
    np.testing.assert_allclose(gl, tgl, rtol=1e-5, atol=1e-9 * np.abs(tgl).max())


def test_gradients_match_finite_differences():
    lat, mlp, R0 = _small_net(seed=5)
    m = synth.material_rgba8(R0, 8, octaves=3, base=2, mips=False)
    targets = synth.ntc_targets(m, 10)
    rng = np.random.default_rng(6)
    ix, iy = rng.integers(0, R0, 64), rng.integers(0, R0, 64)
    _, gm, gl = oracle.ntc_loss_grad(R0, lat, mlp, targets, ix, iy, round_bf16=False)
    # the loss is piecewise smooth (ReLU kinks): a perturbation that moves a sample's
    # pre-activation across zero makes the central difference itself wrong, so at most
    # two of the 40 checks may disagree beyond 1e-4 (and none beyond 1e-2)
    bad = 0
    for idx in rng.choice(6792, 40, replace=False):
        h = np.float32(1e-4)
        p, q = mlp.copy(), mlp.copy()
        p[idx] += h
        q[idx] -= h
        lp = oracle.ntc_loss_grad(R0, lat, p, targets, ix, iy, False)[0]
        lq = oracle.ntc_loss_grad(R0, lat, q, targets, ix, iy, False)[0]
        fd = (lp - lq) / (float(p[idx]) - float(q[idx]))
        err = abs(fd - gm[idx])
        assert err <= 1e-2 * max(abs(fd), 1e-4), (idx, fd, gm[idx])
        bad += err > 1e-4 * max(abs(fd), 1e-4)
    assert bad <= 2
    flat = [g.ravel() for g in lat]
    sizes = np.cumsum([0] + [f.size for f in flat])
    nz = np.flatnonzero(gl)
    # latent perturbations move several samples' pre-activations at once, so kink
    # crossings are more frequent: the check is statistical
    rel = []
    for j in rng.choice(nz, 20, replace=False):
        g = int(np.searchsorted(sizes, j, side="right") - 1)
        k = j - sizes[g]
        lp_, lq_ = [x.copy() for x in lat], [x.copy() for x in lat]
        h = np.float32(1e-4)
        lp_[g].reshape(-1)[k] += h
        lq_[g].reshape(-1)[k] -= h
        dp = float(lp_[g].reshape(-1)[k]) - float(lq_[g].reshape(-1)[k])
        fd = (oracle.ntc_loss_grad(R0, lp_, mlp, targets, ix, iy, False)[0]
              - oracle.ntc_loss_grad(R0, lq_, mlp, targets, ix, iy, False)[0]) / dp
        rel.append(abs(fd - gl[j]) / (abs(fd) + 1e-8))
    rel = np.array(rel)
    assert np.median(rel) < 1e-3 and np.mean(rel < 1e-3) >= 0.8, rel


def test_bf16_backward_rounds_the_gemm_operands():
    # the tensor-core backward feeds dy, dh2 and dh1 to BF16 GEMMs: the oracle's bf16_backward
    # level rounds each once where it is formed (relative error <= 2^-9 per operand)
    lat, mlp, R0 = _small_net(seed=13)
    mlp[2048:2112] = 0.05
    m = synth.material_rgba8(R0, 14, octaves=3, base=2, mips=False)
    targets = synth.ntc_targets(m, 15)
    rng = np.random.default_rng(7)
    ix, iy = rng.integers(0, R0, 256), rng.integers(0, R0, 256)
    l1, g1, d1 = oracle.ntc_loss_grad(R0, lat, mlp, targets, ix, iy, round_bf16=True)
    l2, g2, d2 = oracle.ntc_loss_grad(R0, lat, mlp, targets, ix, iy, round_bf16=True, bf16_backward=True)
    assert l1 == l2                                  # the forward is unchanged
    for a, b in ((g1, g2), (d1, d2)):                # moved, by well under 1e-2 (relative L2)
        d = np.linalg.norm(a - b) / np.linalg.norm(a)
        assert 0 < d < 1e-2, d
    # a zero last layer outputs y = b3 exactly, so db3 is the sum over samples of
    # BF16(2 (b3 - t / 255) / (8 n)), and dh2 = 0 leaves every earlier gradient at zero
    mlp0 = mlp.copy()
    mlp0[6272:6784] = 0.0
    _, g0, d0 = oracle.ntc_loss_grad(R0, lat, mlp0, targets, ix, iy, round_bf16=True, bf16_backward=True)
    t = targets[iy, ix].astype(np.float64) / 255.0
    dy = oracle.round_bf16(2.0 * (mlp0[6784:6792].astype(np.float64) - t) / (8.0 * len(ix)))
    np.testing.assert_allclose(g0[6784:6792], dy.sum(axis=0), rtol=1e-13, atol=0)
    assert not np.any(g0[:6272]) and not np.any(d0)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    p = rng.normal(size=1000)
    g = rng.normal(size=1000)
    p0 = p.copy()
    m, v = np.zeros(1000), np.zeros(1000)
    oracle.adam(p, g, m, v, 1, 0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> step = -lr g / (|g| + eps)
    np.testing.assert_allclose(p - p0, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # a second step with the same gradient keeps the update at -lr sign(g) (constant g)
    p1 = p.copy()
    oracle.adam(p, g, m, v, 2, 0.01)
    np.testing.assert_allclose(p - p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)


def test_decode_rounding_points_and_constant_net():
    # a network whose last layer is zero outputs exactly its bias; the BF16 rounding of
    # the input features is what the decode's features are fed with
    lat, mlp, R0 = _small_net(seed=11)
    mlp[6272:6784] = 0.0
    mlp[6784:6792] = np.arange(8) / 8.0
    nt = oracle.NeuralTexture.inference_form(R0, lat, mlp, "fp16")
    y, rd = oracle.ntc_decode(nt, np.arange(R0), np.arange(R0))
    np.testing.assert_array_equal(y, np.broadcast_to(np.arange(8) / 8.0, y.shape))
    assert np.all((rd >= 0) & (rd <= 1))


def test_fp8_inference_form():
    lat, mlp, R0 = _small_net(seed=12)
    nt = oracle.NeuralTexture.inference_form(R0, lat, mlp, "fp8")
    for g, (codes, sc) in enumerate(zip(nt.grids, nt.scales)):
        vals = oracle.e4m3_value(codes) * sc
        amax = np.abs(lat[g]).max()
        assert abs(sc - amax / 448.0) <= 1e-7 * sc
        # every latent is within half an E4M3 step (relative 2^-4) of its code
        err = np.abs(vals - lat[g])
        assert np.all(err <= np.maximum(np.abs(lat[g]) * 2.0 ** -4, 2.0 ** -10 * sc) + 1e-12)
