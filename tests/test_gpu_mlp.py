"""Surrogate MLP kernels (BF16 tcgen05 GEMMs, FP32 accumulation) against the FP64 MLP oracle.

The oracle is given the network exactly as the tensor cores see it: weights rounded FP64 ->
FP32 master -> BF16, inputs mapped to [-1, 1] and rounded to BF16.  What remains is the
kernels' own BF16 rounding of activations and back-propagated gradients (relative 2^-9 per
element), so the tolerances are:
  forward outputs      relative L2 <= 2e-2, cosine >= 0.999
  loss                 relative <= 1e-2
  gradients            per tensor relative L2 <= 2e-2, cosine >= 0.999
  Adam update          from the kernel's own gradients: the FP32 rounding of the update
"""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2208_04371_b300 import workloads as W

pytestmark = pytest.mark.gpu

LO = np.array([4, 0, 6, 2.0, 0.0, 32], dtype=np.float64)
HI = np.array([40, 10, 30, 12.0, 50.0, 160], dtype=np.float64)


def bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def tensor_core_view(gpu, flat):
    return [(bf16(Wl), bl.astype(np.float32).astype(np.float64))
            for Wl, bl in gpu.mlp_unflatten(flat)]


def mapped_inputs(x):
    x32 = np.asarray(x, dtype=np.float32)
    scale = (2.0 / (HI - LO)).astype(np.float32)
    return bf16((x32 - LO.astype(np.float32)) * scale - np.float32(1.0))


def raw_inputs(seed, n):
    return W.surrogate_inputs(W.SplitMix64(seed), n).astype(np.float32)


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def cos(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b)))


@pytest.mark.parametrize("n", [300, 1, 128, 20000])
def test_forward_matches_oracle(gpu, n):
    flat = W.mlp_init(11, bias_scale=0.1)
    x = raw_inputs(5, n)
    with gpu.Mlp(1, 128, max(512, n), LO, HI) as m:
        m.set_params(0, flat)
        y, est = m.query(x)
    yo = omlp.forward(tensor_core_view(gpu, flat), mapped_inputs(x))[0]
    assert rel(y, yo) <= 2e-2 and cos(y, yo) >= 0.999
    assert np.all(est == 0.0)      # one member: no disagreement


def test_gradients_match_oracle(gpu):
    flat = W.mlp_init(12, bias_scale=0.1)
    B = 256
    x = raw_inputs(6, B)
    t = W.uniform_array(77, B * 512, -1.0, 1.0).reshape(B, 512).astype(np.float32)
    with gpu.Mlp(1, B, 256, LO, HI) as m:
        m.set_params(0, flat)
        loss, g = m.grads(0, x, t)
    lo_, go = omlp.loss_and_grads(tensor_core_view(gpu, flat), mapped_inputs(x), t.astype(np.float64))
    assert loss == pytest.approx(lo_, rel=1e-2)
    for l, ((gW, gb), (oW, ob)) in enumerate(zip(gpu.mlp_unflatten(g), go)):
        for name, a, b in (("W", gW, oW), ("b", gb, ob)):
            assert rel(a, b) <= 2e-2, (l, name, rel(a, b))
            assert cos(a, b) >= 0.999, (l, name, cos(a, b))


def test_adam_step_applies_the_kernel_gradients(gpu):
    flat = W.mlp_init(13, bias_scale=0.1)
    B = 128
    x = raw_inputs(7, B)
    t = W.uniform_array(78, B * 512, -1.0, 1.0).reshape(B, 512).astype(np.float32)
    lr = 1e-3
    with gpu.Mlp(1, B, 128, LO, HI) as m:
        m.set_params(0, flat)
        m.set_adam(lr=lr)
        _, g = m.grads(0, x, t)
        p0 = m.get_params(0)
        m.train_step(0, x, t)
        p1 = m.get_params(0)
    opt = omlp.Adam([(p0, np.zeros(1))], lr=lr)
    expect = opt.step([(p0, np.zeros(1))], [(g.astype(np.float32).astype(np.float64), np.zeros(1))])[0][0]
    assert np.max(np.abs((p1 - p0) - (expect - p0))) <= 1e-5 * lr + 2 * np.spacing(np.float32(1.0)) * np.max(np.abs(p0))


def test_ensemble_mean_disagreement_and_gate(gpu):
    seeds = (21, 22, 23)
    n = 200
    x = raw_inputs(8, n)
    with gpu.Mlp(len(seeds), 128, 256, LO, HI) as m:
        for e, s in enumerate(seeds):
            m.set_params(e, W.mlp_init(s, bias_scale=0.05))
        y, est = m.query(x)
        thr = float(np.median(est))
        flags, cnt = m.gate(est, 1.5, thr)
    ys = [omlp.forward(tensor_core_view(gpu, W.mlp_init(s, bias_scale=0.05)), mapped_inputs(x))[0]
          for s in seeds]
    mean = np.mean(ys, axis=0)
    assert rel(y, mean) <= 2e-2
    d = 0.0
    for yo in ys:
        c = (yo[:, :128] - mean[:, :128]) + 1j * (yo[:, 128:256] - mean[:, 128:256])
        c2 = (yo[:, 256:384] - mean[:, 256:384]) + 1j * (yo[:, 384:] - mean[:, 384:])
        d = np.maximum(d, np.maximum(np.abs(c).max(axis=1), np.abs(c2).max(axis=1)))
    assert rel(est, d) <= 5e-2
    expect = (np.float32(1.5) * est > np.float32(thr)).astype(np.int32)
    assert np.array_equal(flags, expect) and cnt == int(expect.sum())


def test_training_lowers_the_loss(gpu):
    B = 512
    x = raw_inputs(9, B)
    xn = mapped_inputs(x)
    f = np.linspace(0, 1, 128)
    t = np.concatenate([np.cos(np.pi * (xn[:, 5:6] + 1) * f[None] * 3) * (0.3 + 0.2 * xn[:, 0:1]),
                        np.sin(np.pi * (xn[:, 5:6] + 1) * f[None] * 3) * (0.3 + 0.2 * xn[:, 0:1]),
                        np.cos(np.pi * (xn[:, 3:4] + 2) * f[None]) * 0.8,
                        -np.sin(np.pi * (xn[:, 3:4] + 2) * f[None]) * 0.8], axis=1).astype(np.float32)
    with gpu.Mlp(1, B, B, LO, HI) as m:
        m.set_params(0, W.mlp_init(31))
        m.set_adam(lr=1e-3)
        first = m.train_step(0, x, t, want_loss=True)
        for _ in range(300):
            m.train_step(0, x, t)
        last = m.train_step(0, x, t, want_loss=True)
    assert last < 0.05 * first, (first, last)


def test_graph_replayed_fit_equals_step_by_step_training(gpu):
    B, n, steps = 128, 384, 5
    x = raw_inputs(10, n)
    t = W.uniform_array(79, n * 512, -1.0, 1.0).reshape(n, 512).astype(np.float32)
    idx = np.concatenate([np.argsort(W.splitmix64_array(100 + s, n))[:B] for s in range(steps)])
    idx = idx.astype(np.int32)
    lr = np.full(steps, 2e-3, dtype=np.float32)
    flat = W.mlp_init(14, bias_scale=0.1)
    with gpu.Mlp(1, B, 128, LO, HI) as m:
        m.set_params(0, flat)
        m.set_adam(lr=2e-3)
        for s in range(steps):
            rows = idx[s * B:(s + 1) * B]
            m.train_step(0, x[rows], t[rows])
        step_by_step = m.get_params(0)
    with gpu.Mlp(1, B, 128, LO, HI) as m:
        m.set_params(0, flat)
        xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
        m.fit(0, xd, td, torch.from_numpy(idx).cuda(), torch.from_numpy(lr).cuda(), steps)
        m.sync()
        replayed = m.get_params(0)
        # an index outside the training set is reported, not read
        bad = torch.from_numpy(np.full(B, n, dtype=np.int32)).cuda()
        m.fit(0, xd, td, bad, torch.from_numpy(lr[:1]).cuda(), 1)
        with pytest.raises(gpu.YFError) as e:
            m.sync()
        assert e.value.code == gpu.E_INVALID
    assert np.array_equal(step_by_step, replayed)
