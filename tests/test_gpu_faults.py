"""Failure detection without faulting a GPU: a device wait on a flag nothing sets gives up and
reports YF_E_TIMEOUT; an allocation the device cannot satisfy reports YF_E_OOM; both leave the
context usable.  Runs repeat bit for bit (fixed-order reductions), so a race would show up as
a difference between two identical runs."""
import numpy as np
import pytest

from paper_2208_04371_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _small_run(gpu):
    p = W.config_small_fp64()
    with gpu.Grid(p, prec=gpu.FP32) as g:
        g.step(300)
        g.sync()
        return g.fields(), g.port_dfts()


def test_device_wait_times_out_and_context_survives(gpu):
    gpu.bounded_wait_check(True, 1.0)            # flag set beforehand: returns at once
    with pytest.raises(gpu.YFError) as e:
        gpu.bounded_wait_check(False, 0.2)       # nothing ever sets it: gives up
    assert e.value.code == gpu.E_TIMEOUT
    f, _ = _small_run(gpu)                       # the context still runs kernels
    assert np.isfinite(f).all() and np.abs(f).max() > 0


def test_oversized_grid_reports_oom_and_context_survives(gpu):
    # 4000^3 FP64 cells need about 3 TB of fields: the allocation fails on the host side of
    # the driver, nothing runs on the GPU
    with pytest.raises(gpu.YFError) as e:
        gpu.grid_create(4000, 4000, 4000, 5e-6, 5e-6, 5e-6, prec=gpu.FP64)
    assert e.value.code == gpu.E_OOM
    f, _ = _small_run(gpu)
    assert np.isfinite(f).all()


def test_identical_runs_are_bitwise_identical(gpu):
    f1, (V1, I1) = _small_run(gpu)
    f2, (V2, I2) = _small_run(gpu)
    assert np.array_equal(f1, f2) and np.array_equal(V1, V2) and np.array_equal(I1, I2)
