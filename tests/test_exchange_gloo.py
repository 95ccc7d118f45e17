"""One all-at-once solve sharded over gloo CPU ranks through the two all-to-all
transposes (space-first and the paper's time-first order, eq. 3.8).

Each rank runs its stages on its own slab only; the stages are written here
from the factorisation of Section 3.3 with the oracle's building blocks (sine
matrices, Laplacian eigenvalues, C_omega, the principal root), and the
gathered result must equal the oracle's single-process sine-basis solve."""
import datetime
import math
import os
import queue
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bhcp_inputs as bi
from paper_2107_06381_gb300 import exchange as X

SPACE_CASES = [
    # (dim, M, L, T, nt, form)
    (2, (8, 16), 1.0, 0.1, 6, 0),
    (2, (16, 8), math.pi, 1.0, 9, 1),
    (3, (4, 8, 4), 1.0, 0.05, 5, 0),
    (1, (13,), 1.0, 0.1, 4, 1),            # 12 modes, 4 levels: uneven slabs
]
TIME_CASES = [
    (1, (12,), 1.0, 0.1, 7, 0),
    (1, (9,), math.pi, 1.0, 5, 1),
    (2, (8, 4), 1.0, 0.1, 6, 1),
]
ALPHA = 1e-3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _grid(case):
    dim, M, L, T, nt, form = case
    return bi.Grid(dim, M, L, T, nt), form


def _apply_axes(a, grid, mats):
    """Apply mats[d] along spatial axis d of an (n_levels, *grid.shape) array."""
    for d in range(grid.dim):
        ax = grid.dim - d
        a = np.moveaxis(np.tensordot(mats[d], np.moveaxis(a, ax, 0), axes=(1, 0)), 0, ax)
    return a


def _space_stages(grid, form):
    import torch
    import oracle as O
    S = [O.sine_matrix(m - 1) for m in grid.M]
    Sinv = [O.sine_matrix(m - 1) * (2.0 / m) for m in grid.M]
    lam = np.zeros(grid.shape)
    for d in range(grid.dim):
        shape = [1] * grid.dim
        shape[grid.dim - 1 - d] = grid.M[d] - 1
        lam = lam + O.dst_eigenvalues(grid.M[d], grid.L).reshape(shape)
    lam = lam.ravel()                                   # x fastest, as the columns
    tau = grid.tau
    C = O.c_omega(grid.nt, O.omega_of(form, ALPHA, tau)) / tau

    def dst(rows):
        a = rows.numpy().reshape((-1,) + grid.shape)
        return torch.from_numpy(np.ascontiguousarray(_apply_axes(a, grid, S).reshape(rows.shape)))

    def time_solve(cols, m0, m1):
        s = cols.numpy()
        out = np.empty_like(s)
        for j in range(m1 - m0):                        # per sine mode: (C_omega/tau + lambda) y = s
            out[:, j] = np.linalg.solve(C + lam[m0 + j] * np.eye(grid.nt), s[:, j])
        return torch.from_numpy(out)

    def idst(rows):
        a = rows.numpy().reshape((-1,) + grid.shape)
        return torch.from_numpy(np.ascontiguousarray(_apply_axes(a, grid, Sinv).reshape(rows.shape)))

    return dst, time_solve, idst


def _time_stages(grid, form):
    """Steps (a)-(c) of eq. (3.8): V^{-1} = F Gamma, D = sqrt(N_t) F Gamma C(:,1),
    V = Gamma^{-1} F*, with F the unitary DFT (theta = exp(2 pi i / N_t))."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import torch
    import oracle as O
    from oracle.qbvm_oracle import principal_root
    nt, tau = grid.nt, grid.tau
    om = O.omega_of(form, ALPHA, tau)
    k = np.arange(nt)
    Fm = np.exp(2j * np.pi * np.outer(k, k) / nt) / math.sqrt(nt)
    gam = principal_root(om, nt) ** k
    Vinv = Fm * gam[None, :]
    V = (1.0 / gam)[:, None] * Fm.conj().T
    d = math.sqrt(nt) * (Vinv @ O.c_omega(nt, om)[:, 0])
    Lap = O.laplacian(grid.dim, grid.M, grid.L).tocsc()
    I = sp.identity(Lap.shape[0], format="csc")

    def step_a(cols):
        return torch.from_numpy(Vinv @ cols.numpy().astype(complex))

    def step_b(rows, k0, k1):
        s = rows.numpy()
        out = np.empty_like(s)
        for i, j in enumerate(range(k0, k1)):
            out[i] = spla.splu(((d[j] / tau) * I - Lap).tocsc()).solve(s[i])
        return torch.from_numpy(out)

    def step_c(cols):
        return torch.from_numpy(V @ cols.numpy())

    return step_a, step_b, step_c


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=120))
    out = {}
    # transposes alone, real and complex, with ranks that own no rows
    for n_t, n_x in [(5, 7), (2, 9), (7, 2), (1, 1)]:
        rng = np.random.default_rng(100 + n_t * 10 + n_x)
        A = rng.standard_normal((n_t, n_x)) + 1j * rng.standard_normal((n_t, n_x))
        for cplx in (False, True):
            G = torch.from_numpy(A if cplx else A.real.copy())
            lo, hi = X.slab(n_t, rank, world)
            c0, c1 = X.slab(n_x, rank, world)
            cols = X.rows_to_columns(G[lo:hi].contiguous(), n_t, n_x)
            back = X.columns_to_rows(cols, n_t, n_x)
            out[("t", n_t, n_x, cplx)] = (bool(torch.equal(cols, G[:, c0:c1])),
                                          bool(torch.equal(back, G[lo:hi])))
    for i, case in enumerate(SPACE_CASES):
        grid, form = _grid(case)
        F = bi.random_general_rhs(grid, seed=40 + i).reshape(grid.nt, grid.Nx)
        lo, hi = X.slab(grid.nt, rank, world)
        y = X.solve_space_first(torch.from_numpy(np.ascontiguousarray(F[lo:hi])), grid.nt, grid.Nx,
                                *_space_stages(grid, form))
        out[("s", i)] = (lo, hi, y.numpy())
    for i, case in enumerate(TIME_CASES):
        grid, form = _grid(case)
        F = bi.random_general_rhs(grid, seed=60 + i).reshape(grid.nt, grid.Nx)
        c0, c1 = X.slab(grid.Nx, rank, world)
        y = X.solve_time_first(torch.from_numpy(np.ascontiguousarray(F[:, c0:c1])), grid.nt, grid.Nx,
                               *_time_stages(grid, form))
        out[("c", i)] = (c0, c1, y.numpy())
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def _run(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    try:
        while len(res) < world:                 # a rank that dies ends the test at once
            try:
                r, out = q.get(timeout=2)
                res[r] = out
            except queue.Empty:
                dead = [p.exitcode for p in procs if p.exitcode not in (None, 0)]
                assert not dead, f"a rank exited with {dead}"
    finally:
        for p in procs:
            if p.is_alive() and len(res) < world:
                p.kill()
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.fixture(scope="module", params=[2, 3], ids=lambda w: f"world{w}")
def ranks(request):
    return request.param, _run(request.param)


def test_transposes_are_exact_and_invert(ranks):
    world, res = ranks
    for r in range(world):
        keys = [k for k in res[r] if k[0] == "t"]
        assert len(keys) == 8
        for key in keys:
            fwd, back = res[r][key]
            assert fwd and back, (r, key)


@pytest.mark.parametrize("i", range(len(SPACE_CASES)))
def test_space_first_sharded_solve_matches_oracle(ranks, i):
    import oracle as O
    world, res = ranks
    grid, form = _grid(SPACE_CASES[i])
    F = bi.random_general_rhs(grid, seed=40 + i)
    y = np.empty((grid.nt, grid.Nx))
    for r in range(world):
        lo, hi, part = res[r][("s", i)]
        assert (lo, hi) == X.slab(grid.nt, r, world)
        y[lo:hi] = part
    want = O.solve_spectral(grid, form, ALPHA, F)
    assert O.rel_l2(y, want) <= 1e-12


@pytest.mark.parametrize("i", range(len(TIME_CASES)))
def test_time_first_sharded_solve_matches_oracle(ranks, i):
    import oracle as O
    world, res = ranks
    grid, form = _grid(TIME_CASES[i])
    F = bi.random_general_rhs(grid, seed=60 + i)
    y = np.empty((grid.nt, grid.Nx), dtype=complex)
    for r in range(world):
        c0, c1, part = res[r][("c", i)]
        y[:, c0:c1] = part
    want = O.solve_spectral(grid, form, ALPHA, F)
    assert np.abs(y.imag).max() <= 1e-10 * np.abs(y.real).max()
    assert O.rel_l2(y.real, want) <= 1e-10


def test_slabs_partition_contiguously_and_balance():
    for n in [0, 1, 5, 7, 256, 255 * 255]:
        for world in [1, 2, 3, 8]:
            s = X.slabs(n, world)
            assert s[0][0] == 0 and s[-1][1] == n
            assert all(s[r][1] == s[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in s]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        X.slab(4, 2, 2)


def test_exchange_bytes_counts_off_rank_blocks():
    # 256 levels x 255^2 modes over 8 ranks: each rank keeps 1/8 of its rows
    b = X.exchange_bytes(256, 255 * 255, 8)
    assert len(b) == 8
    total = 256 * 255 * 255 * 8
    assert abs(sum(b) - total * 7 / 8) <= 8 * 256 * 8
    assert X.exchange_bytes(16, 16, 1) == [0]
