"""Learned S-parameter surrogate with FDTD fallback.

The paper obtains each line's S-matrix from full FDTD runs (Sec. II-A).  This module trains
an ensemble of small networks (yfmlp.h) on S-matrices that the batched FDTD solver computes
for seeded line descriptors, answers new descriptors from the ensemble where its members
agree, and sends the rest back to the solver:

  descriptor (width, thickness, substrate height [cells], eps_r, sigma [S/m], length [cells])
  -> network outputs [Re S11, Im S11, Re S21, Im S21] x 128 frequencies (50-ohm S, Eq. 5-6)
  -> disagreement est = max over members, entries and frequencies of |S_m - S_mean|
  -> accepted if scale * est <= 1e-2, else solved by FDTD.

`scale` is calibrated on held-out FDTD solves: the smallest factor with which scale * est
bounds the realised error |S_mean - S_fdtd| (max over entries and frequencies) for the
chosen fraction of those solves.  Every arithmetic step (network, loss, Adam, ensemble, gate,
FDTD, S extraction) runs in the library's kernels; this module stages data and loops.
"""
from __future__ import annotations

import time
from typing import Optional

import numpy as np

from . import workloads as W
from . import yf

THRESHOLD = 1e-2


def s_to_outputs(S: np.ndarray) -> np.ndarray:
    """S [F, 2, 2] complex -> [Re S11 | Im S11 | Re S21 | Im S21] float32 (4 F)."""
    return np.concatenate([S[:, 0, 0].real, S[:, 0, 0].imag, S[:, 1, 0].real,
                           S[:, 1, 0].imag]).astype(np.float32)


def outputs_to_s(y: np.ndarray):
    """[..., 4 F] -> (S11, S21) complex [..., F]."""
    F = y.shape[-1] // 4
    return y[..., :F] + 1j * y[..., F:2 * F], y[..., 2 * F:3 * F] + 1j * y[..., 3 * F:]


def s_error(y: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Max over S11, S21 and frequencies of the complex difference, per row."""
    a11, a21 = outputs_to_s(np.asarray(y, dtype=np.float64))
    b11, b21 = outputs_to_s(np.asarray(t, dtype=np.float64))
    return np.maximum(np.abs(a11 - b11).max(axis=-1), np.abs(a21 - b21).max(axis=-1))


def fdtd_solve(descs: np.ndarray, nsteps: int = 5000, chunk: int = 512, stream=None,
               log=None) -> tuple:
    """Targets [n, 512] for each descriptor through the batched FDTD solver (FP32 fields, FP64
    spectra, 50-ohm S from the uniform-line extraction), and the wall time in seconds."""
    n = len(descs)
    out = np.zeros((n, 4 * 128), dtype=np.float32)
    t0 = time.perf_counter()
    for s in range(0, n, chunk):
        probs = [W.surrogate_line(d, nsteps=nsteps) for d in descs[s:s + chunk]]
        with yf.Batch(probs, prec=yf.FP32, stream=stream) as b:
            b.step(nsteps)
            b.sync()
            for q in range(len(probs)):
                out[s + q] = s_to_outputs(b.sparams(q)["S"])
        if log:
            log(f"fdtd {s + len(probs)}/{n} {time.perf_counter() - t0:.1f}s")
    return out, time.perf_counter() - t0


def _perm(seed: int, n: int) -> np.ndarray:
    return np.argsort(W.splitmix64_array(seed, n))


class Surrogate:
    def __init__(self, members: int = 4, train_batch: int = 512, max_query: int = 65536,
                 seed: int = 0x5EED, stream=None):
        self.mlp = yf.Mlp(members, train_batch, max_query, W.SURROGATE_LO, W.SURROGATE_HI, stream)
        self.members, self.batch, self.seed = members, train_batch, seed
        for e in range(members):
            self.mlp.set_params(e, W.mlp_init(seed + 7919 * e))
        self.scale = 1.0

    def fit(self, x: np.ndarray, t: np.ndarray, epochs: int, lr: float = 1e-3,
            lr_end: float = 2e-5, log=None) -> list:
        """Adam on every member, each with its own seeded shuffle per epoch; the learning rate
        decays geometrically from lr to lr_end.  One graph-replayed yf_mlp_fit call per member.
        Returns the last batch loss per member."""
        import torch
        xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
        td = torch.from_numpy(np.ascontiguousarray(t, dtype=np.float32)).cuda()
        n = len(x)
        per = n // self.batch
        steps = per * epochs
        sched = torch.from_numpy((lr * (lr_end / lr) ** (np.arange(steps) / max(steps - 1, 1)))
                                 .astype(np.float32)).cuda()
        losses = []
        for e in range(self.members):
            idx = np.concatenate([_perm(self.seed * 31 + e * 1000003 + ep, n)[:per * self.batch]
                                  for ep in range(epochs)]).astype(np.int32)
            idx_d = torch.from_numpy(idx).cuda()
            self.mlp.fit(e, xd, td, idx_d, sched, steps)
            losses.append(self.mlp.sync())
            if log:
                log(f"member {e}: {steps} steps, last batch loss {losses[-1]:.3e}")
        return losses

    def predict(self, x: np.ndarray):
        """(ensemble mean [n, 512], disagreement [n])"""
        return self.mlp.query(np.ascontiguousarray(x, dtype=np.float32))

    def calibrate(self, x: np.ndarray, t: np.ndarray, coverage: float = 0.95) -> float:
        """Set scale so that scale * est >= realised error on `coverage` of the given
        held-out solves."""
        y, est = self.predict(x)
        err = s_error(y, t)
        ratio = err / np.maximum(est.astype(np.float64), 1e-12)
        self.scale = float(np.quantile(ratio, coverage))
        return self.scale

    def gate(self, est: np.ndarray):
        return self.mlp.gate(est, self.scale, THRESHOLD)

    def answer(self, x: np.ndarray, nsteps: int = 5000, stream=None) -> dict:
        """S outputs for every descriptor: the ensemble where the gate accepts it, the batched
        FDTD solver where it does not."""
        t0 = time.perf_counter()
        y, est = self.predict(x)
        flags, nflag = self.gate(est)
        t1 = time.perf_counter()
        out = y.copy()
        fb = np.nonzero(flags)[0]
        fdtd_s = 0.0
        if len(fb):
            out[fb], fdtd_s = fdtd_solve(x[fb], nsteps=nsteps, stream=stream)
        return {"y": out, "est": est, "flags": flags, "fallback": int(nflag),
                "surrogate_s": t1 - t0, "fdtd_s": fdtd_s}

    def close(self):
        self.mlp.close()
