"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only *generates* inputs: stencil matrices M, K0, K1 in CSR form, the
parameter / shift lists and the right-hand-side blocks.  It contains none of the
method's arithmetic (no assembly of A(p, s), no SPAI, no update, no Krylov solve),
so that the CPU oracle and the CUDA path can both consume it without sharing any of
the computation they are compared on.

Conventions
-----------
* CSR triplets are ``(rowptr int32[n+1], colind int32[nnz], val float64[nnz])`` with
  strictly increasing column indices inside each row.
* Grids are ordered lexicographically with x fastest: ``idx = x + nx*(y + ny*z)``.
  Boundary conditions are homogeneous Dirichlet: couplings to points outside the
  grid are dropped.
* Right-hand-side blocks are ``(n, s)`` float64 arrays in column-major (Fortran)
  order, i.e. column i is contiguous.
* Random streams: ``SeedSequence(seed).spawn(3)`` gives independent children used
  for, in order, the K1 diagonal, the right-hand sides and the parameter draws.
"""

from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------------------
# stencil patterns
# --------------------------------------------------------------------------------------


def _offsets(kind: str):
    if kind == "5pt":
        return [(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    if kind == "7pt":
        return [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    if kind == "27pt":
        return [(dx, dy, dz) for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3)]
    raise ValueError(f"unknown stencil {kind!r}")


def stencil_csr(dims, kind: str, center: float, off, face_only_off=None):
    """CSR matrix of a constant-coefficient stencil on a 2D/3D grid.

    ``dims`` is (nx, ny) or (nx, ny, nz).  ``center`` is the diagonal value, ``off``
    the value on every non-centre stencil entry.  If ``face_only_off`` is given, only
    face neighbours (|dx|+|dy|+|dz| == 1) are kept and receive that value.
    """
    dims = tuple(int(d) for d in dims)
    if len(dims) == 2:
        nx, ny = dims
        nz = 1
    else:
        nx, ny, nz = dims
    n = nx * ny * nz
    offs = _offsets(kind)
    if len(dims) == 2:
        offs = [o for o in offs if o[2] == 0]
    if face_only_off is not None:
        offs = [o for o in offs if sum(abs(c) for c in o) <= 1]
    # ascending linear offset == ascending column index inside each row
    offs = sorted(offs, key=lambda o: o[0] + nx * (o[1] + ny * o[2]))
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    cols = np.empty((n, len(offs)), dtype=np.int64)
    vals = np.empty((n, len(offs)), dtype=np.float64)
    mask = np.empty((n, len(offs)), dtype=bool)
    for t, (dx, dy, dz) in enumerate(offs):
        xx, yy, zz = x + dx, y + dy, z + dz
        mask[:, t] = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        cols[:, t] = idx + dx + nx * (dy + ny * dz)
        if (dx, dy, dz) == (0, 0, 0):
            vals[:, t] = center
        else:
            vals[:, t] = off if face_only_off is None else face_only_off
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colind = cols[mask].astype(np.int32)
    val = vals[mask].copy()
    return rowptr.astype(np.int32), colind, val


def diag_csr(d):
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    return (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d.copy())


def csr_to_dense(csr, n):
    rowptr, colind, val = csr
    D = np.zeros((n, n))
    for i in range(n):
        for q in range(rowptr[i], rowptr[i + 1]):
            D[i, colind[q]] += val[q]
    return D


def dense_to_csr(D, keep=None):
    """CSR of dense ``D``; ``keep`` (bool array) selects the structural pattern (default D != 0)."""
    D = np.asarray(D, dtype=np.float64)
    n = D.shape[0]
    if keep is None:
        keep = D != 0
    rowptr = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        c = np.nonzero(keep[i])[0]
        cols.append(c)
        vals.append(D[i, c])
        rowptr[i + 1] = rowptr[i] + len(c)
    colind = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    val = np.concatenate(vals).astype(np.float64) if vals else np.zeros(0)
    return rowptr, colind, val


# --------------------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------------------


@dataclass
class Workload:
    """Terms of the affine system A(p, s) = c_M(s) M + c_K0(s) K0 + c_K1(p, s) K1 plus RHS."""

    name: str
    n: int
    M: tuple
    K0: tuple
    K1: tuple
    B: np.ndarray                 # (n, nrhs), Fortran order
    params: list                  # parameter values p (base first)
    shifts: list                  # shift values s
    restart: int
    tol: float
    dims: tuple = ()
    extra: dict = field(default_factory=dict)
    alpha: float = 0.05           # Rayleigh damping of the workload: D(p) = alpha M + beta K(p)
    beta: float = 0.01

    @property
    def terms(self):
        return [self.M, self.K0, self.K1]


def _streams(seed):
    ss = np.random.SeedSequence(seed)
    return [np.random.default_rng(c) for c in ss.spawn(3)]


def grid_workload(dims, kind, *, seed=0, nrhs=4, params=None, shifts=(1.0,), restart=30,
                  tol=1e-8, nparams=None, m_off=0.1, name=None):
    """FEM-like stencil workload: K0 Laplacian, K1 = U[0.5,1.5] diagonal, M = stencil (diag 1).

    For the 27-point stencil, K1 additionally carries face couplings of -0.1 and M uses
    off-diagonal 0.02 (the large 3D workload); 5/7-point stencils use M off-diagonal 0.1.
    """
    rng_k1, rng_b, rng_p = _streams(seed)
    npts = {"5pt": 5, "7pt": 7, "27pt": 27}[kind]
    n = int(np.prod(dims))
    K0 = stencil_csr(dims, kind, float(npts - 1), -1.0)
    M = stencil_csr(dims, kind, 1.0, m_off)
    d = rng_k1.uniform(0.5, 1.5, size=n)
    if kind == "27pt":
        faces = stencil_csr(dims, kind, 0.0, 0.0, face_only_off=-0.1)
        K1 = (faces[0], faces[1], faces[2].copy())
        # put the random diagonal on the centre entries of the face stencil
        for_rows = np.repeat(np.arange(n), np.diff(faces[0]))
        centre = faces[1] == for_rows
        K1[2][centre] = d
    else:
        K1 = diag_csr(d)
    B = np.asfortranarray(rng_b.standard_normal((n, nrhs)))
    if params is None:
        params = sorted(rng_p.uniform(0.1, 1.0, size=nparams).tolist())
    return Workload(name=name or f"{kind}-{'x'.join(map(str, dims))}", n=n, M=M, K0=K0, K1=K1,
                    B=B, params=list(params), shifts=list(shifts), restart=restart, tol=tol,
                    dims=tuple(dims))


def plain_2d_32(seed=0):
    """2D 32x32 5-point grid, n=1024: p in {0.1..0.5}, s=1, 4 RHS, GMRES(30), tol 1e-8."""
    return grid_workload((32, 32), "5pt", seed=seed, nrhs=4, params=[0.1, 0.2, 0.3, 0.4, 0.5],
                         shifts=[1.0], restart=30, tol=1e-8, name="2d-32x32-5pt")


def grid3d_7pt(side=64, seed=0, nrhs=8, nparams=20, shifts=(0.5, 1.0, 2.0), restart=50):
    """3D side^3 7-point grid (side=64: n=262,144): 20 p ~ U[0.1,1] sorted, s in {0.5,1,2}, 8 RHS."""
    return grid_workload((side, side, side), "7pt", seed=seed, nrhs=nrhs, nparams=nparams,
                         shifts=shifts, restart=restart, tol=1e-8, name=f"3d-{side}^3-7pt")


def grid3d_27pt(side=128, seed=0, nrhs=16, nparams=50, restart=30):
    """3D side^3 27-point grid (side=128: n=2,097,152), 50 p in [0.1,2.0], s=1, 16 RHS."""
    w = grid_workload((side, side, side), "27pt", seed=seed, nrhs=nrhs,
                      params=np.linspace(0.1, 2.0, nparams).tolist(), shifts=[1.0],
                      restart=restart, tol=1e-8, m_off=0.02, name=f"3d-{side}^3-27pt")
    return w


def appendix1_matrix(s: float, p: float):
    """A(s, p) = s I - diag(A1(p), A2, A3, A4) of the worked example (Appendix I), n = 1006.

    A1(p) = [[-1, p], [-p, -1]], A2 = [[-1, 200], [-200, -1]], A3 = [[-1, 400], [-400, -1]],
    A4 = diag(1, ..., 1000).  Returned as CSR with the 2x2 blocks stored in full.
    """
    n = 1006
    D = np.zeros((n, n))
    for b, w in ((0, p), (2, 200.0), (4, 400.0)):
        blk = np.array([[-1.0, w], [-w, -1.0]])
        D[b:b + 2, b:b + 2] = s * np.eye(2) - blk
    k = np.arange(1, 1001, dtype=np.float64)
    D[6 + np.arange(1000), 6 + np.arange(1000)] = s - k
    keep = np.zeros((n, n), dtype=bool)
    for b in (0, 2, 4):
        keep[b:b + 2, b:b + 2] = True
    keep[np.arange(6, n), np.arange(6, n)] = True
    return dense_to_csr(D, keep)


def random_sparse(n, density, seed, *, symmetric_pattern=False, diag_shift=None):
    """Random nonsymmetric sparse matrix with a full nonzero diagonal (seeded).

    Off-diagonal entries are N(0,1) at Bernoulli(density) positions; the diagonal is
    ``diag_shift`` (default: 1 + row abs-sum, i.e. diagonally dominant) plus noise.
    """
    rng = np.random.default_rng(seed)
    keep = rng.random((n, n)) < density
    if symmetric_pattern:
        keep = keep | keep.T
    np.fill_diagonal(keep, True)
    D = np.where(keep, rng.standard_normal((n, n)), 0.0)
    np.fill_diagonal(D, 0.0)
    if diag_shift is None:
        dg = 1.0 + np.abs(D).sum(axis=1) * 0.5 + rng.uniform(0.0, 1.0, n)
    else:
        dg = np.full(n, float(diag_shift))
    D[np.arange(n), np.arange(n)] = dg
    return dense_to_csr(D, keep), D


def bordered_sparse(n, density, seed, border_rows=1):
    """``random_sparse`` with its first ``border_rows`` rows full (a bordered matrix, as a
    constraint row or a global coupling gives): every column meets those rows, so a least-
    squares problem whose row set contains one of them sees all n columns as neighbours.
    The border entries are N(0,1) * 0.1; the diagonal stays dominant."""
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(1)[0])
    (_, _, _), D = random_sparse(n, density, seed)
    keep = D != 0
    keep[:border_rows, :] = True
    D[:border_rows, :] = np.where(D[:border_rows, :] != 0, D[:border_rows, :],
                                  0.1 * rng.standard_normal((border_rows, n)))
    D[np.arange(border_rows), np.arange(border_rows)] += 0.1 * n
    return dense_to_csr(D, keep), D


def rhs_block(n, s, seed):
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(3)[1])
    return np.asfortranarray(rng.standard_normal((n, s)))


def batched_2d(nsys=256, seed=0):
    """The many-small-systems workload: nsys 2D 5-point grids with sides ~ U{48..256}
    (n = 2,304 .. 65,536), system i seeded with 1000 + i, its parameter p ~ U[0.1, 1] and
    shift 1, 4 right-hand sides; even-numbered systems take the SPAI pattern of A, odd ones
    that of A^2 (recorded in ``extra["pattern"]``)."""
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(5)[4])
    sides = rng.integers(48, 257, size=nsys)
    ps = rng.uniform(0.1, 1.0, size=nsys)
    out = []
    for i in range(nsys):
        w = grid_workload((int(sides[i]), int(sides[i])), "5pt", seed=1000 + i, nrhs=4, params=[float(ps[i])])
        w.extra["pattern"] = "A" if i % 2 == 0 else "A2"
        out.append(w)
    return out


SERVE_SIDES = [round(24 + 72 * i / 15) for i in range(16)]  # 24 ... 96: n = 13,824 ... 884,736


def serving_pool(seed=100):
    """The serving workload's pool of 16 3D 7-point grids (sides 24 .. 96), 8 RHS each."""
    return [grid_workload((d, d, d), "7pt", seed=seed + i, nrhs=8, params=[0.5]) for i, d in enumerate(SERVE_SIDES)]


def serving_trace(rate, seconds, nsys, seed=0):
    """Poisson arrivals at `rate` per second for `seconds`: (t, system, p, s, nrhs).  70 % of
    the requests lie within 0.05 of an already-served (system, s, p); the others draw a
    system, p ~ U[0.1, 1] and s in {0.5, 1, 2}; nrhs in {1, 4, 8}."""
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(4)[3])
    out, seen, t = [], [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            return out
        if seen and rng.random() < 0.7:
            sy, p0, s = seen[int(rng.integers(len(seen)))]
            p = float(np.clip(p0 + rng.uniform(-0.05, 0.05), 0.1, 1.0))
        else:
            sy, p, s = int(rng.integers(nsys)), float(rng.uniform(0.1, 1.0)), float(rng.choice([0.5, 1.0, 2.0]))
        seen.append((sy, p, s))
        out.append((t, sy, p, s, int(rng.choice([1, 4, 8]))))
