"""What the learned surrogate gains over FDTD alone, end to end on the GPU.

Lines are drawn from a reduced box of the descriptor ranges (width 4-16, thickness 0-4,
substrate 6-12 cells, eps_r 2-6, sigma 0-20 S/m, length 32-64 cells) so that the whole
workflow fits in about a minute:
  1. 2048 FDTD solves (batched solver, 4000 steps): 1536 to train, 256 to calibrate the
     gate, 256 to test;
  2. a 4-member ensemble trained by the library's kernels (20000 graph-replayed Adam steps);
  3. the test queries answered by the ensemble where the calibrated gate accepts them and by
     FDTD where it does not.
Error = max over S11, S21 and the 128 frequencies of |S - S_fdtd| (complex)."""
import time

import numpy as np
import pytest

from paper_2208_04371_b300 import workloads as W

pytestmark = pytest.mark.gpu

LO = np.array([4, 0, 6, 2.0, 0.0, 32])
HI = np.array([16, 4, 12, 6.0, 20.0, 64])
NSTEPS = 4000


def _descriptors(n):
    u = np.stack([W.uniform_array(900 + k, n, 0.0, 1.0) for k in range(6)], axis=1)
    x = LO + u * (HI - LO)
    x[:, [0, 1, 2, 5]] = np.round(x[:, [0, 1, 2, 5]])
    return x.astype(np.float32)


def test_surrogate_with_fdtd_fallback_beats_fdtd_alone(gpu):
    from paper_2208_04371_b300 import surrogate as S
    x = _descriptors(2048)
    t, _ = S.fdtd_solve(x, nsteps=NSTEPS, chunk=1024)
    tr, cal, te = slice(0, 1536), slice(1536, 1792), slice(1792, 2048)
    sur = S.Surrogate(members=4, train_batch=256, max_query=4096)
    try:
        untrained = np.median(S.s_error(sur.predict(x[te])[0], t[te]))
        sur.fit(x[tr], t[tr], epochs=20000 // 6)
        y, est = sur.predict(x[te])
        err = S.s_error(y, t[te])
        # the network learned the map: 20x below its untrained error and under 2e-2 typically
        assert np.median(err) < 0.05 * untrained and np.median(err) < 2e-2
        # disagreement tracks the realised error
        assert np.corrcoef(err, est)[0, 1] > 0.5
        sur.calibrate(x[cal], t[cal])

        t0 = time.perf_counter()
        ans = sur.answer(x[te], nsteps=NSTEPS)
        t_answer = time.perf_counter() - t0
        t0 = time.perf_counter()
        S.fdtd_solve(x[te], nsteps=NSTEPS)
        t_fdtd = time.perf_counter() - t0
    finally:
        sur.close()
    acc = ans["flags"] == 0
    final_err = S.s_error(ans["y"], t[te])
    print(f"accepted {acc.mean():.3f}, accepted error p90 {np.quantile(err[acc], 0.9):.4f} "
          f"max {err[acc].max():.4f}, answer {t_answer:.2f}s vs FDTD {t_fdtd:.2f}s")
    assert acc.mean() >= 0.4                        # most queries need no solve
    assert np.quantile(err[acc], 0.9) <= 1e-2       # the gate keeps accepted answers in budget
    assert err[acc].max() <= 3e-2
    assert np.all(final_err[~acc] == 0.0)           # fallback answers are the FDTD solves
    assert np.quantile(final_err, 0.95) <= 1e-2
    assert t_answer < t_fdtd
