"""The z-slab decomposition a multi-GPU single-line solve would use, checked on CPU ranks.

One line is never split across GPUs in this build: every box has one GPU, and several GPUs
run replicas. The exchange that a split would need is still pinned down here. Cut the grid
at node plane K along z; rank 0 owns node planes k < K (E_x, E_y, H_z) and half planes
k + 1/2 < K (H_x, H_y, E_z), rank 1 the rest. Per step the ranks exchange two tangential
components, one plane in each direction:
  before the H half-step: rank 1 -> rank 0   E_x, E_y at node plane K
                           (H_x, H_y at half plane K - 1/2 take dE/dz across the cut);
  before the E half-step: rank 0 -> rank 1   H_x, H_y at half plane K - 1/2
                           (E_x, E_y at node plane K take dH/dz across the cut).
Two `gloo` ranks step a PEC cavity from random fields with a plain numpy Yee update and must
match the unsplit run bit for bit. The unsplit numpy run must match the FP64 oracle to
roundoff.
"""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import yee
from paper_2208_04371_b300 import workloads as W

NX, NY, NZ, CUT = 10, 9, 14, 6
DX, DY, DZ = 1e-3, 0.8e-3, 1.1e-3
MU0, EPS0 = 1.25663706212e-6, 8.8541878128e-12


def _problem():
    return W.Problem(nx=NX, ny=NY, nz=NZ, dx=DX, dy=DY, dz=DZ, courant=0.95,
                     ids=np.zeros((NZ, NY, NX), np.uint8), eps_r=np.array([1.0]),
                     sigma=np.array([0.0]), mu_r=np.array([1.0]),
                     is_pec=np.array([0], np.uint8), bc=(0,) * 6, pml_cells=0)


def _initial():
    f = W.random_fields((NZ + 1, NY + 1, NX + 1), seed=0xD15C)
    ex, ey, ez, hx, hy, hz = f
    # PEC walls: tangential E zero; positions outside each component's range zero
    ex[:, :, NX:] = 0; ex[:, [0, NY], :] = 0; ex[[0, NZ], :, :] = 0
    ey[:, NY:, :] = 0; ey[:, :, [0, NX]] = 0; ey[[0, NZ], :, :] = 0
    ez[NZ:, :, :] = 0; ez[:, :, [0, NX]] = 0; ez[:, [0, NY], :] = 0
    hx[NZ:, :, :] = 0; hx[:, NY:, :] = 0
    hy[NZ:, :, :] = 0; hy[:, :, NX:] = 0
    hz[:, NY:, :] = 0; hz[:, :, NX:] = 0
    return f


def _h_step(f, db, k0, k1):
    """H on half planes k in [k0, k1) (H_x, H_y) and node planes k in [k0, k1) (H_z)."""
    ex, ey, ez, hx, hy, hz = f
    rdx, rdy, rdz = 1.0 / DX, 1.0 / DY, 1.0 / DZ
    ks = slice(k0, min(k1, NZ))
    kp = slice(k0 + 1, min(k1, NZ) + 1)
    hx[ks, :NY, :] = hx[ks, :NY, :] - db * ((ez[ks, 1:NY + 1, :] - ez[ks, :NY, :]) * rdy
                                            - (ey[kp, :NY, :] - ey[ks, :NY, :]) * rdz)
    hy[ks, :, :NX] = hy[ks, :, :NX] - db * ((ex[kp, :, :NX] - ex[ks, :, :NX]) * rdz
                                            - (ez[ks, :, 1:NX + 1] - ez[ks, :, :NX]) * rdx)
    kn = slice(k0, min(k1, NZ + 1))
    hz[kn, :NY, :NX] = hz[kn, :NY, :NX] - db * ((ey[kn, :NY, 1:NX + 1] - ey[kn, :NY, :NX]) * rdx
                                                - (ex[kn, 1:NY + 1, :NX] - ex[kn, :NY, :NX]) * rdy)


def _e_step(f, cb, k0, k1):
    """E on node planes k in [k0, k1) (E_x, E_y) and half planes k in [k0, k1) (E_z)."""
    ex, ey, ez, hx, hy, hz = f
    rdx, rdy, rdz = 1.0 / DX, 1.0 / DY, 1.0 / DZ
    ks = slice(max(k0, 1), min(k1, NZ))
    km = slice(max(k0, 1) - 1, min(k1, NZ) - 1)
    ex[ks, 1:NY, :NX] = 1.0 * ex[ks, 1:NY, :NX] + cb * ((hz[ks, 1:NY, :NX] - hz[ks, :NY - 1, :NX]) * rdy
                                                         - (hy[ks, 1:NY, :NX] - hy[km, 1:NY, :NX]) * rdz)
    ey[ks, :NY, 1:NX] = 1.0 * ey[ks, :NY, 1:NX] + cb * ((hx[ks, :NY, 1:NX] - hx[km, :NY, 1:NX]) * rdz
                                                         - (hz[ks, :NY, 1:NX] - hz[ks, :NY, :NX - 1]) * rdx)
    kz = slice(k0, min(k1, NZ))
    ez[kz, 1:NY, 1:NX] = 1.0 * ez[kz, 1:NY, 1:NX] + cb * ((hy[kz, 1:NY, 1:NX] - hy[kz, 1:NY, :NX - 1]) * rdx
                                                          - (hx[kz, 1:NY, 1:NX] - hx[kz, :NY - 1, 1:NX]) * rdy)


def _coeffs():
    dt = yee.courant_dt(DX, DY, DZ, 0.95)
    return dt, dt / MU0, (dt / EPS0) / 1.0


def _run_unsplit(nsteps):
    dt, db, cb = _coeffs()
    f = _initial()
    for _ in range(nsteps):
        _h_step(f, db, 0, NZ + 1)
        _e_step(f, cb, 0, NZ + 1)
    return f


def _rank(rank, world, port, nsteps, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dt, db, cb = _coeffs()
    f = _initial()
    k0, k1 = (0, CUT) if rank == 0 else (CUT, NZ + 1)
    for _ in range(nsteps):
        # E_x, E_y at node plane CUT: rank 1 -> rank 0
        if rank == 1:
            dist.send(torch.from_numpy(np.ascontiguousarray(f[0:2, CUT])), dst=0)
        else:
            buf = torch.zeros((2, NY + 1, NX + 1), dtype=torch.float64)
            dist.recv(buf, src=1)
            f[0:2, CUT] = buf.numpy()
        _h_step(f, db, k0, k1)
        # H_x, H_y at half plane CUT - 1/2: rank 0 -> rank 1
        if rank == 0:
            dist.send(torch.from_numpy(np.ascontiguousarray(f[3:5, CUT - 1])), dst=1)
        else:
            buf = torch.zeros((2, NY + 1, NX + 1), dtype=torch.float64)
            dist.recv(buf, src=0)
            f[3:5, CUT - 1] = buf.numpy()
        _e_step(f, cb, k0, k1)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), f)
    dist.destroy_process_group()


def test_unsplit_numpy_step_matches_the_oracle():
    f = _run_unsplit(60)
    ref = yee.run(_problem(), nsteps=60, fields_in=_initial(), want_fields=True)["fields"]
    assert np.linalg.norm((f - ref).ravel()) <= 1e-13 * np.linalg.norm(ref.ravel())


def test_two_gloo_ranks_match_the_unsplit_run_bitwise(tmp_path):
    nsteps = 60
    port = 29600 + os.getpid() % 1000
    mp.spawn(_rank, args=(2, port, nsteps, str(tmp_path)), nprocs=2, join=True)
    whole = _run_unsplit(nsteps)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    # node-plane components (E_x, E_y, H_z) below / from the cut, half-plane ones likewise
    for c in range(6):
        assert np.array_equal(r0[c, :CUT], whole[c, :CUT]), c
        assert np.array_equal(r1[c, CUT:], whole[c, CUT:]), c
