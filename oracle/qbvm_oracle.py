"""CPU FP64 oracle for the PinT quasi-boundary value methods (arXiv 2107.06381).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library (no kernels, tables, helpers or headers); it takes the same seeded
inputs from ``bhcp_inputs`` and nothing else.

Contents (all plain, slow and obviously checkable against the paper):

* ``laplacian``             Section 2: the Dirichlet 3/5/7-point finite-difference
                            Laplacian Delta_h on interior nodes.
* ``omega_of``, ``rhs_block0``
                            Section 3.1 (PinT-QBVM, omega = -1/alpha, first RHS
                            block g/(tau alpha)) and Section 3.2 (PinT-MQBVM,
                            omega = -tau/alpha, first block g/alpha).
* ``assemble_pint``         the all-at-once matrices of eqs. (3.3)/(3.6), built
                            block row by block row as printed.
* ``assemble_original``     the original QBVM / MQBVM matrices A_h, B_h of
                            Sections 2.1/2.2 (comparison methods).
* ``solve_sparse_lu``       O1, the oracle of record: sparse direct LU of the
                            assembled system (SuperLU through scipy).
* ``solve_dense``           O2: dense LU of the same matrix (tiny grids).
* ``solve_pint_three_step`` the paper's Section 3.3 three-step diagonalisation
                            with explicit V = Gamma^{-1} F*, D and per-frequency
                            sparse solves, in the paper's order (eq. 3.8).
* ``solve_spectral``        O3: exact solve in the sine eigenbasis of Delta_h
                            (dense sine matrices, no FFT) with the per-mode
                            cyclic backward-Euler recurrence solved in closed
                            form; exact for any right-hand side.
* ``residual``              f - A y for the assembled matrix.
* ``alpha_apriori``         Section 5 rule: alpha = delta (PinT-QBVM), tau*delta
                            (PinT-MQBVM).

Conventions: ``nt`` = N_t = N + 1 time levels, tau = T/(nt - 1); arrays have
shape (nt, n_z, n_y, n_x) with x fastest, which is the paper's vec ordering of
y_h = (y^0; y^1; ...; y^N) (Section 2).
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

PQ = 0   # PinT-QBVM   (Section 3.1)
PM = 1   # PinT-MQBVM  (Section 3.2)

__all__ = [
    "PQ", "PM", "laplacian_1d", "laplacian", "omega_of", "rhs_block0", "delta_rhs",
    "assemble_pint", "assemble_original", "c_omega", "solve_sparse_lu", "solve_dense",
    "solve_pint_three_step", "solve_spectral", "residual", "rel_residual",
    "alpha_apriori", "dst_eigenvalues", "sine_matrix", "rel_l2",
]


# ------------------------------------------------------------------ operators

def laplacian_1d(M: int, L: float) -> sp.csr_matrix:
    """Section 2: central second difference with homogeneous Dirichlet values on
    the M-1 interior nodes of (0, L), h = L/M: (y_{i-1} - 2 y_i + y_{i+1}) / h^2."""
    n = M - 1
    h = L / M
    main = np.full(n, -2.0 / h ** 2)
    off = np.full(n - 1, 1.0 / h ** 2)
    return sp.diags([off, main, off], [-1, 0, 1], shape=(n, n), format="csr")


def laplacian(dim: int, M, L: float) -> sp.csr_matrix:
    """Section 2: the 5-point (2D) Laplacian, adapted to 1D (3-point) and 3D
    (7-point), on interior nodes ordered with x fastest."""
    Ms = tuple(M) if hasattr(M, "__len__") else (M,) * dim
    ops = [laplacian_1d(m, L) for m in Ms]              # x, y, z
    eyes = [sp.identity(m - 1, format="csr") for m in Ms]
    total = None
    for d in range(dim):
        # kron ordering: slowest axis first -> (z, y, x); axis d acts where its op sits
        factors = []
        for e in reversed(range(dim)):
            factors.append(ops[e] if e == d else eyes[e])
        term = factors[0]
        for f in factors[1:]:
            term = sp.kron(term, f, format="csr")
        total = term if total is None else total + term
    return total.tocsr()


def omega_of(form: int, alpha: float, tau: float) -> float:
    """Section 3.1: omega = -1/alpha (PinT-QBVM); Section 3.2: omega = -tau/alpha
    (PinT-MQBVM)."""
    if alpha <= 0:
        raise ValueError("alpha must be positive")
    return -1.0 / alpha if form == PQ else -tau / alpha


def rhs_block0(form: int, alpha: float, tau: float, g: np.ndarray) -> np.ndarray:
    """First block of the right-hand side: g/(tau alpha) in eq. (3.3) (PinT-QBVM),
    g/alpha in eq. (3.6) (PinT-MQBVM); every other block is zero."""
    return g / (tau * alpha) if form == PQ else g / alpha


def delta_rhs(grid, form: int, alpha: float, g: np.ndarray) -> np.ndarray:
    """The full all-at-once right-hand side (nt, *shape) with only block 0 nonzero."""
    F = np.zeros(grid.full_shape)
    F[0] = rhs_block0(form, alpha, grid.tau, np.asarray(g).reshape(grid.shape))
    return F


def c_omega(nt: int, omega: float) -> np.ndarray:
    """Section 3.3: C_omega, unit diagonal, -1 on the subdiagonal, -omega in the
    top-right corner (dense, nt x nt)."""
    C = np.eye(nt) - np.eye(nt, k=-1)
    C[0, nt - 1] = -omega
    return C


def assemble_pint(grid, form: int, alpha: float) -> sp.csr_matrix:
    """The all-at-once matrix of eq. (3.3) (form PQ, omega=-1/alpha) or
    eq. (3.6) (form PM, omega=-tau/alpha), assembled block row by block row:

      row 0:       [-Lap + I/tau, 0, ..., 0, -omega I/tau]
      row n >= 1:  [..., -I/tau (column n-1), -Lap + I/tau (column n), ...]
    """
    tau = grid.tau
    om = omega_of(form, alpha, tau)
    Lap = laplacian(grid.dim, grid.M, grid.L)
    Nx = Lap.shape[0]
    I = sp.identity(Nx, format="csr")
    diag_block = (-Lap + I / tau).tocsr()
    nt = grid.nt
    blocks = [[None] * nt for _ in range(nt)]
    for n in range(nt):
        blocks[n][n] = diag_block
        if n >= 1:
            blocks[n][n - 1] = -I / tau
    if nt >= 2:
        blocks[0][nt - 1] = (-om / tau) * I
    return sp.bmat(blocks, format="csr")


def assemble_original(grid, method: str, alpha: float) -> sp.csr_matrix:
    """The original systems of Section 2: A_h (QBVM, eq. 2.3: first block row
    [alpha I, 0, ..., I]) and B_h (MQBVM, eq. 2.6: [alpha I/tau, -alpha I/tau,
    0, ..., I]); the other block rows are the backward Euler rows.  The matching
    right-hand side has g in block 0."""
    tau = grid.tau
    Lap = laplacian(grid.dim, grid.M, grid.L)
    Nx = Lap.shape[0]
    I = sp.identity(Nx, format="csr")
    nt = grid.nt
    blocks = [[None] * nt for _ in range(nt)]
    for n in range(1, nt):
        blocks[n][n] = (-Lap + I / tau).tocsr()
        blocks[n][n - 1] = -I / tau
    if method == "qbvm":
        blocks[0][0] = alpha * I
        blocks[0][nt - 1] = I
    elif method == "mqbvm":
        blocks[0][0] = (alpha / tau) * I
        if nt == 2:                       # y^1 is y^N: the two blocks add up
            blocks[0][1] = (-alpha / tau) * I + I
        else:
            blocks[0][1] = (-alpha / tau) * I
            blocks[0][nt - 1] = I
    else:
        raise ValueError(method)
    return sp.bmat(blocks, format="csr")


# ------------------------------------------------------------------- solvers

def _as_vec(F: np.ndarray) -> np.ndarray:
    return np.asarray(F, dtype=np.float64).reshape(-1)


def solve_sparse_lu(grid, form: int, alpha: float, F: np.ndarray) -> np.ndarray:
    """O1: assemble eq. (3.3)/(3.6) and solve it with a sparse direct LU."""
    A = assemble_pint(grid, form, alpha).tocsc()
    lu = spla.splu(A)
    return lu.solve(_as_vec(F)).reshape(grid.full_shape)


def solve_dense(grid, form: int, alpha: float, F: np.ndarray) -> np.ndarray:
    """O2: dense LU (partial pivoting) of the same assembled matrix."""
    A = assemble_pint(grid, form, alpha).toarray()
    return np.linalg.solve(A, _as_vec(F)).reshape(grid.full_shape)


def solve_original(grid, method: str, alpha: float, g: np.ndarray) -> np.ndarray:
    """Sparse LU of the original QBVM/MQBVM system with f_h = (g, 0, ..., 0)."""
    A = assemble_original(grid, method, alpha).tocsc()
    f = np.zeros(grid.full_shape)
    f[0] = np.asarray(g).reshape(grid.shape)
    return spla.splu(A).solve(f.reshape(-1)).reshape(grid.full_shape)


def principal_root(omega: float, nt: int) -> complex:
    """omega^{1/N_t} with the principal branch (for omega < 0 this is
    |omega|^{1/N_t} e^{i pi / N_t})."""
    return complex(omega) ** (1.0 / nt)


def solve_pint_three_step(grid, form: int, alpha: float, F: np.ndarray,
                          return_imag: bool = False):
    """Section 3.3, eq. (3.8), in the paper's order and notation.

    With F_hat = mat(f) (N_x x N_t, column n = time level n):
      Step (a): S1 = F_hat (V^{-1})^T, V^{-1} = F Gamma_omega,
      Step (b): S2(:, j) = (d_j/tau I - Lap)^{-1} S1(:, j) for every j,
      Step (c): y = vec(S2 V^T),      V = Gamma_omega^{-1} F*,
    where F is the unitary DFT matrix with theta = exp(2 pi i / N_t),
    Gamma_omega = diag(omega^{k/N_t}) and D = diag(sqrt(N_t) F Gamma_omega C(:,1)).
    Dense V, V^{-1}; sparse LU per frequency (the paper uses a sparse direct
    solver in Step (b)).
    """
    nt = grid.nt
    tau = grid.tau
    om = omega_of(form, alpha, tau)
    k = np.arange(nt)
    Fm = np.exp(2j * np.pi * np.outer(k, k) / nt) / math.sqrt(nt)
    gam = principal_root(om, nt)
    Gam = np.diag(gam ** k)
    Gam_inv = np.diag(gam ** (-k.astype(np.float64)))
    V = Gam_inv @ Fm.conj().T
    Vinv = Fm @ Gam
    d = math.sqrt(nt) * (Fm @ Gam @ c_omega(nt, om)[:, 0])
    Fhat = np.asarray(F, dtype=np.float64).reshape(nt, -1).T          # N_x x N_t
    S1 = Fhat @ Vinv.T
    Lap = laplacian(grid.dim, grid.M, grid.L).tocsc()
    I = sp.identity(Lap.shape[0], format="csc")
    S2 = np.empty_like(S1)
    for j in range(nt):
        Aj = (d[j] / tau) * I - Lap
        S2[:, j] = spla.splu(Aj.tocsc()).solve(S1[:, j])
    Y = S2 @ V.T                                                      # N_x x N_t
    y = Y.T.reshape(grid.full_shape)
    if return_imag:
        return y.real, float(np.abs(y.imag).max())
    return y.real


def sine_matrix(n: int) -> np.ndarray:
    """S_{jk} = sin(pi j k / (n + 1)), j, k = 1..n: the DST-I matrix; the columns
    are the eigenvectors of the 1D Dirichlet Laplacian."""
    j = np.arange(1, n + 1)
    return np.sin(np.pi * np.outer(j, j) / (n + 1))


def dst_eigenvalues(M: int, L: float) -> np.ndarray:
    """Eigenvalues of -Delta_h in 1D for sine mode k: (4/h^2) sin^2(k pi/(2M))."""
    h = L / M
    return (4.0 / h ** 2) * np.sin(np.arange(1, M) * np.pi / (2 * M)) ** 2


def _apply_axis(S: np.ndarray, c: np.ndarray, ax: int) -> np.ndarray:
    return np.moveaxis(np.tensordot(S, np.moveaxis(c, ax, 0), axes=(1, 0)), 0, ax)


def solve_spectral(grid, form: int, alpha: float, F: np.ndarray, levels=None) -> np.ndarray:
    """O3: the exact solution of eq. (3.3)/(3.6) in the sine eigenbasis.

    Delta_h = S diag(-Lambda) S^{-1} with dense sine matrices per axis
    (S^{-1} = (2/M) S).  In that basis every mode l decouples into the scalar
    cyclic system of the backward-Euler rows and the corner row:
        (1 + tau Lambda) y^0 - omega y^N = tau f^0,
        (1 + tau Lambda) y^n - y^{n-1}   = tau f^n   (n = 1..N),
    whose solution, with r = 1/(1 + tau Lambda) and q the n>=1 recurrence
    started from zero (q^N = sum_n r^{N-n+1} tau f^n), is
        y^0 = (tau f^0 + omega q^N) / (1 + tau Lambda - omega r^N),
        y^n = r (y^{n-1} + tau f^n).
    No FFT is used anywhere, so this shares nothing with an FFT-based path.
    ``levels`` (optional) restricts the returned time levels (the inverse DST
    is then applied to those levels only); F may then also be given as the
    single level g when it is a delta right-hand side of shape grid.shape.
    """
    tau = grid.tau
    om = omega_of(form, alpha, tau)
    nt = grid.nt
    F = np.asarray(F, dtype=np.float64)
    if F.size == grid.Nx:                       # delta right-hand side given as level 0 only
        F0 = F.reshape((1,) + grid.shape)
        Fh = np.zeros(grid.full_shape)
        Fh[0] = F0[0]
    else:
        Fh = F.reshape(grid.full_shape).copy()
    lam = np.zeros(grid.shape)
    for d in range(grid.dim):
        M = grid.M[d]
        ax = grid.dim - d          # axis in the (nt, ...) array
        Fh = _apply_axis(sine_matrix(M - 1), Fh, ax)
        shape = [1] * grid.dim
        shape[grid.dim - 1 - d] = M - 1
        lam = lam + dst_eigenvalues(M, grid.L).reshape(shape)
    r = 1.0 / (1.0 + tau * lam)
    q = np.zeros(grid.shape)
    for n in range(1, nt):
        q = r * (q + tau * Fh[n])
    rN = r ** (nt - 1)
    Y = np.empty_like(Fh)
    Y[0] = (tau * Fh[0] + om * q) / (1.0 + tau * lam - om * rN)
    for n in range(1, nt):
        Y[n] = r * (Y[n - 1] + tau * Fh[n])
    if levels is not None:
        Y = Y[list(levels)]
    for d in range(grid.dim):
        M = grid.M[d]
        ax = grid.dim - d
        Y = _apply_axis(sine_matrix(M - 1) * (2.0 / M), Y, ax)
    return Y


def residual(grid, form: int, alpha: float, y: np.ndarray, F: np.ndarray) -> np.ndarray:
    """f - A y with A the assembled eq. (3.3)/(3.6) matrix."""
    A = assemble_pint(grid, form, alpha)
    return (_as_vec(F) - A @ _as_vec(y)).reshape(grid.full_shape)


def rel_residual(grid, form: int, alpha: float, y: np.ndarray, F: np.ndarray) -> float:
    r = residual(grid, form, alpha, y, F)
    return float(np.linalg.norm(r.ravel()) / np.linalg.norm(_as_vec(F)))


def alpha_apriori(form: int, delta: float, tau: float) -> float:
    """Section 5: alpha = delta for PinT-QBVM and alpha = tau*delta for PinT-MQBVM
    (E_0 unknown in Theorem 4.1's choice alpha = delta/E_0 resp. tau delta/E_0)."""
    return delta if form == PQ else tau * delta


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_2 / ||b||_2."""
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(np.asarray(a).ravel() - b) / np.linalg.norm(b))
