"""The one-exchange design for sharding ONE all-at-once solve across ranks.

The all-at-once unknowns form an N_t x N_x array (time level n = row, spatial
unknown or sine mode = column; row-major, the layout of the device solve).
The factorisation of Section 3.3 makes every stage independent along one of
the two axes:

* space-first order (the DST-I diagonalises -Delta_h): the forward and
  inverse DSTs act on each time level alone, the scalar omega-circulant time
  solve on each sine mode alone;
* the paper's time-first order (eq. 3.8): Steps (a) and (c) act along time
  for each spatial unknown alone, Step (b) on each frequency alone.

So a rank that owns a contiguous slab of rows for one stage and a contiguous
slab of columns for the other needs exactly one all-to-all transpose in each
direction and nothing else.  This module holds the partition, the two
transposes (``torch.distributed.all_to_all_single``, any backend with uneven
splits) and the two stage drivers; the stages themselves are callables, so the
same driver runs host stages over gloo or device stages over NCCL.
"""
from __future__ import annotations

from typing import Callable, List, Tuple


def slab(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous share [lo, hi) of n items for `rank` of `world`: the first
    n mod world ranks take one more item; ranks past n get empty slabs."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("need n >= 0 and 0 <= rank < world")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def slabs(n: int, world: int) -> List[Tuple[int, int]]:
    return [slab(n, r, world) for r in range(world)]


def _world(group):
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def _as_real(x):
    """Complex tensors travel as their (re, im) pairs; returns (view, was_complex)."""
    import torch
    if x.is_complex():
        return torch.view_as_real(x), True
    return x, False


def rows_to_columns(x, n_rows: int, n_cols: int, group=None):
    """Row slab -> column slab.  `x` is this rank's rows [lo, hi) of the
    n_rows x n_cols array (shape (hi - lo, n_cols)); the result is all n_rows
    rows of this rank's columns [clo, chi) (shape (n_rows, chi - clo)).
    One all_to_all_single; each rank sends (hi - lo)(chi_s - clo_s) elements
    to rank s."""
    import torch
    import torch.distributed as dist
    rank, world = _world(group)
    xr, cplx = _as_real(x)
    tail = tuple(xr.shape[2:])
    rows, cols = slabs(n_rows, world), slabs(n_cols, world)
    lo, hi = rows[rank]
    if tuple(xr.shape[:2]) != (hi - lo, n_cols):
        raise ValueError(f"rank {rank}: expected rows ({hi - lo}, {n_cols}), got {tuple(xr.shape[:2])}")
    if world == 1:
        return x.contiguous()
    e = 1
    for t in tail:
        e *= t
    send = torch.cat([xr[:, c0:c1].reshape(-1) for c0, c1 in cols]) if n_cols else xr.reshape(-1)
    c0, c1 = cols[rank]
    nc = c1 - c0
    recv = torch.empty(n_rows * nc * e, dtype=xr.dtype, device=xr.device)
    dist.all_to_all_single(recv, send.contiguous(),
                           output_split_sizes=[(r1 - r0) * nc * e for r0, r1 in rows],
                           input_split_sizes=[(hi - lo) * (d1 - d0) * e for d0, d1 in cols],
                           group=group)
    out = recv.view((n_rows, nc) + tail)     # row blocks arrive in rank order = row order
    return torch.view_as_complex(out) if cplx else out


def columns_to_rows(y, n_rows: int, n_cols: int, group=None):
    """Column slab -> row slab, the inverse of ``rows_to_columns``: `y` holds
    all rows of this rank's columns (shape (n_rows, chi - clo)); the result is
    this rank's rows [lo, hi) over all columns (shape (hi - lo, n_cols))."""
    import torch
    import torch.distributed as dist
    rank, world = _world(group)
    yr, cplx = _as_real(y)
    tail = tuple(yr.shape[2:])
    rows, cols = slabs(n_rows, world), slabs(n_cols, world)
    c0, c1 = cols[rank]
    nc = c1 - c0
    if tuple(yr.shape[:2]) != (n_rows, nc):
        raise ValueError(f"rank {rank}: expected columns ({n_rows}, {nc}), got {tuple(yr.shape[:2])}")
    if world == 1:
        return y.contiguous()
    e = 1
    for t in tail:
        e *= t
    lo, hi = rows[rank]
    send = yr.contiguous().reshape(-1)       # row blocks of a row-major slab are contiguous
    recv = torch.empty((hi - lo) * n_cols * e, dtype=yr.dtype, device=yr.device)
    dist.all_to_all_single(recv, send,
                           output_split_sizes=[(hi - lo) * (d1 - d0) * e for d0, d1 in cols],
                           input_split_sizes=[(r1 - r0) * nc * e for r0, r1 in rows],
                           group=group)
    parts, off = [], 0
    for d0, d1 in cols:
        k = (hi - lo) * (d1 - d0) * e
        parts.append(recv[off:off + k].view((hi - lo, d1 - d0) + tail))
        off += k
    out = torch.cat(parts, dim=1) if parts else recv.view((hi - lo, n_cols) + tail)
    return torch.view_as_complex(out.contiguous()) if cplx else out


def solve_space_first(f_rows, n_t: int, n_x: int,
                      dst: Callable, time_solve: Callable, idst: Callable, group=None):
    """Space-first all-at-once solve sharded over the ranks of `group`.

    f_rows            this rank's time levels [lo, hi) of F (shape (hi - lo, N_x))
    dst(rows)         forward DST-I of every level in the slab (same shape)
    time_solve(cols, m0, m1)
                      the scalar omega-circulant solve of sine modes [m0, m1)
                      over all N_t levels (shape (N_t, m1 - m0))
    idst(rows)        inverse DST-I of every level in the slab
    Returns this rank's time levels of y.  Exchanges: one transpose each way.
    """
    rank, world = _world(group)
    m0, m1 = slab(n_x, rank, world)
    s = dst(f_rows)
    s = rows_to_columns(s, n_t, n_x, group)
    s = time_solve(s, m0, m1)
    s = columns_to_rows(s, n_t, n_x, group)
    return idst(s)


def solve_time_first(f_cols, n_t: int, n_x: int,
                     step_a: Callable, step_b: Callable, step_c: Callable, group=None):
    """The paper's time-first order (eq. 3.8) sharded over the ranks of `group`.

    f_cols            all N_t levels of this rank's spatial unknowns [x0, x1)
    step_a(cols)      Step (a): the scaled time DFT of every column (complex)
    step_b(rows, k0, k1)
                      Step (b): the shifted spatial solves of frequencies [k0, k1)
                      over all spatial unknowns (shape (k1 - k0, N_x))
    step_c(cols)      Step (c): the inverse scaled time DFT of every column
    Returns all levels of this rank's spatial unknowns of y.
    """
    rank, world = _world(group)
    k0, k1 = slab(n_t, rank, world)
    z = step_a(f_cols)
    z = columns_to_rows(z, n_t, n_x, group)
    z = step_b(z, k0, k1)
    z = rows_to_columns(z, n_t, n_x, group)
    return step_c(z)


def exchange_bytes(n_t: int, n_x: int, world: int, elem_bytes: int = 8) -> List[int]:
    """Bytes each rank sends to the OTHER ranks in one transpose (the same in
    both directions): sum over s != r of |rows_r| |cols_s| elem_bytes."""
    rows, cols = slabs(n_t, world), slabs(n_x, world)
    out = []
    for r in range(world):
        nr = rows[r][1] - rows[r][0]
        out.append(sum(nr * (c1 - c0) for s, (c0, c1) in enumerate(cols) if s != r) * elem_bytes)
    return out
