"""Seeded synthetic matrices shaped like the paper's block-structured Jacobians.

The paper's test matrices (RANS Jacobians of the DPW3 wing, SuiteSparse
collections) are not available, so every input here is synthetic.  The shapes
follow what Section 4.2 states about the turbulent Navier-Stokes Jacobians:
ell = d+2 (incompressible) or d+3 (compressible) unknowns per mesh node, a
structurally symmetric block pattern and about 14 block entries per block row
in 3-D.

This module only draws random numbers and lays them out as CSR arrays.  It
holds none of the preconditioner's arithmetic, so both the CUDA path and the
CPU oracle can be fed from it.  ``numpy.random.default_rng`` (PCG64) makes
every matrix a pure function of its arguments.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class CSR:
    """A pointwise sparse matrix: 0-based, columns ascending and unique."""
    n: int
    rowptr: np.ndarray  # int64[n+1]
    colind: np.ndarray  # int32[nnz]
    val: np.ndarray     # float64[nnz]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.colind, self.rowptr), shape=(self.n, self.n))

    def dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        a[rows, self.colind] = self.val
        return a

    def matvec(self, x: np.ndarray) -> np.ndarray:
        return self.to_scipy() @ x


def _from_scipy(m, meta=None) -> CSR:
    m = m.tocsr()
    m.sort_indices()
    return CSR(m.shape[0], m.indptr.astype(np.int64), m.indices.astype(np.int32),
               m.data.astype(np.float64), dict(meta or {}))


def _expand_blocks(n_nodes: int, ell: int, nptr: np.ndarray, nidx: np.ndarray,
                   blocks: np.ndarray, keep: np.ndarray | None) -> CSR:
    """Lay out dense ell x ell node blocks as a pointwise CSR matrix.

    ``nptr``/``nidx`` is the node adjacency (including the node itself, columns
    ascending); ``blocks[k]`` is the ell x ell block of adjacency entry k and
    ``keep[k]`` its scalar keep mask (None keeps everything).
    """
    deg = np.diff(nptr).astype(np.int64)
    nblk = int(nptr[-1])
    row_node = np.repeat(np.arange(n_nodes, dtype=np.int64), deg)
    t_local = np.arange(nblk, dtype=np.int64) - nptr[row_node]
    i = np.arange(ell, dtype=np.int64)[None, :, None]
    j = np.arange(ell, dtype=np.int64)[None, None, :]
    # CSR position of (block k, i, j) when no entry is dropped: row node*ell+i
    # starts at nptr[node]*ell^2 + i*deg*ell; block k contributes columns
    # t_local*ell .. +ell within that row.
    pos = (nptr[row_node][:, None, None] * ell * ell + i * deg[row_node][:, None, None] * ell
           + t_local[:, None, None] * ell + j)
    total = nblk * ell * ell
    vals = np.empty(total, dtype=np.float64)
    cols = np.empty(total, dtype=np.int32)
    vals[pos.ravel()] = blocks.reshape(-1)
    cols[pos.ravel()] = (nidx.astype(np.int64)[:, None, None] * ell + j
                         + 0 * i).astype(np.int32).reshape(-1)
    row_len_full = np.repeat(deg * ell, ell)
    if keep is None:
        rowptr = np.zeros(n_nodes * ell + 1, dtype=np.int64)
        np.cumsum(row_len_full, out=rowptr[1:])
        return CSR(n_nodes * ell, rowptr, cols, vals)
    kmask = np.empty(total, dtype=bool)
    kmask[pos.ravel()] = keep.reshape(-1)
    rows_full = np.repeat(np.arange(n_nodes * ell, dtype=np.int64), row_len_full)
    counts = np.bincount(rows_full[kmask], minlength=n_nodes * ell)
    rowptr = np.zeros(n_nodes * ell + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n_nodes * ell, rowptr, cols[kmask], vals[kmask])


def _adjacency_from_pairs(n_nodes: int, pairs: np.ndarray):
    """Symmetric node adjacency with self loops, columns ascending."""
    a = np.concatenate([pairs[:, 0], pairs[:, 1], np.arange(n_nodes)])
    b = np.concatenate([pairs[:, 1], pairs[:, 0], np.arange(n_nodes)])
    order = np.lexsort((b, a))
    a, b = a[order], b[order]
    nptr = np.zeros(n_nodes + 1, dtype=np.int64)
    np.cumsum(np.bincount(a, minlength=n_nodes), out=nptr[1:])
    return nptr, b.astype(np.int64)


def _scramble(m: CSR, seed: int) -> CSR:
    """Symmetric random permutation Q A Q^T of the scalar unknowns."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    q = rng.permutation(m.n)
    s = m.to_scipy()[q][:, q]
    out = _from_scipy(sp.csr_matrix(s), m.meta)
    out.meta["scramble"] = q  # new row k is old row q[k]
    return out


def grid_7pt(nx: int = 10, ny: int = 10, nz: int = 10, ell: int = 5, seed: int = 0,
             scramble: bool = False) -> CSR:
    """Structured 3-D grid, 7-point node connectivity, exact dense ell x ell blocks.

    Nodes are numbered lexicographically (x fastest).  Off-diagonal block
    entries are N(0, 0.1^2); diagonal blocks are N(0, 1) + 8 I (nonsymmetric).
    With ``scramble`` the scalar unknowns are symmetrically permuted by a
    seeded random permutation so that the blocks are no longer contiguous.
    """
    rng = np.random.default_rng(seed)
    nn = nx * ny * nz
    idx = np.arange(nn).reshape(nz, ny, nx)
    pairs = []
    for axis in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(0, -1)
        hi[axis] = slice(1, None)
        pairs.append(np.stack([idx[tuple(lo)].ravel(), idx[tuple(hi)].ravel()], axis=1))
    pairs = np.concatenate(pairs) if pairs else np.zeros((0, 2), np.int64)
    nptr, nidx = _adjacency_from_pairs(nn, pairs)
    nblk = int(nptr[-1])
    blocks = rng.standard_normal((nblk, ell, ell)) * 0.1
    row_node = np.repeat(np.arange(nn), np.diff(nptr))
    diag = np.nonzero(row_node == nidx)[0]
    blocks[diag] = rng.standard_normal((nn, ell, ell)) + 8.0 * np.eye(ell)
    m = _expand_blocks(nn, ell, nptr, nidx, blocks, None)
    m.meta.update(kind="grid7", nodes=nn, ell=ell, seed=seed,
                  node_of_row=np.repeat(np.arange(nn), ell))
    return _scramble(m, seed + 7919) if scramble else m


def _morton30(pts: np.ndarray) -> np.ndarray:
    q = np.minimum((pts * 1024).astype(np.int64), 1023)

    def spread(v):
        v = v & 0x3FF
        v = (v | (v << 16)) & 0x030000FF
        v = (v | (v << 8)) & 0x0300F00F
        v = (v | (v << 4)) & 0x030C30C3
        v = (v | (v << 2)) & 0x09249249
        return v

    return spread(q[:, 0]) | (spread(q[:, 1]) << 1) | (spread(q[:, 2]) << 2)


def geometric(n_nodes: int, ell: int = 6, seed: int = 0, approx: bool = True,
              drop_p: float = 0.1, noise_var: float = 1e-3, degree: float = 15.0,
              dominance: float | None = None, ill_frac: float = 0.0,
              ill_cond: float = 1e6, scramble: bool = False) -> CSR:
    """Random geometric 3-D node graph with ell unknowns per node.

    Points are uniform in the periodic unit cube; two nodes are coupled when
    their torus distance is below r = (3*degree/(4*pi*N))^(1/3), so a node has
    ``degree`` neighbours on average.  Nodes are numbered in 30-bit Morton
    order.  Block values follow ``grid_7pt``.  With ``approx`` every scalar
    entry except the scalar diagonal is dropped with probability ``drop_p`` and
    every kept entry gets additive N(0, noise_var) noise, so node blocks are
    only approximately dense.

    ``dominance`` (e.g. 1.5) replaces each diagonal block by a dense
    D_a = s_a U diag(sig) V^T with random orthogonal U, V, sig ~ U[1, 2] and
    s_a = dominance * sum_b ||A_ab||_F / min(sig), so that
    sigma_min(D_a) = dominance * sum_b ||A_ab||_F (block diagonal dominance in
    the 2-norm); a seeded fraction ``ill_frac`` of nodes instead get
    sig = (1, ..., 1, 1/ill_cond) and s_a = dominance * sum_b ||A_ab||_F, so
    kappa_2(D_a) = ill_cond exactly.
    """
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    pts = rng.random((n_nodes, 3))
    order = np.argsort(_morton30(pts), kind="stable")
    pts = pts[order]
    r = (3.0 * degree / (4.0 * np.pi * n_nodes)) ** (1.0 / 3.0)
    if n_nodes > 1:
        pairs = cKDTree(pts, boxsize=1.0).query_pairs(min(r, 0.4999), output_type="ndarray")
    else:
        pairs = np.zeros((0, 2), dtype=np.int64)
    nptr, nidx = _adjacency_from_pairs(n_nodes, pairs.astype(np.int64))
    nblk = int(nptr[-1])
    row_node = np.repeat(np.arange(n_nodes, dtype=np.int64), np.diff(nptr))
    is_diag = row_node == nidx
    blocks = rng.standard_normal((nblk, ell, ell)) * 0.1
    diag = np.nonzero(is_diag)[0]
    blocks[diag] = rng.standard_normal((n_nodes, ell, ell)) + 8.0 * np.eye(ell)
    keep = None
    eye = np.eye(ell, dtype=bool)
    if approx:
        keep = rng.random((nblk, ell, ell)) >= drop_p
        keep[diag] |= eye[None]
        blocks += rng.standard_normal((nblk, ell, ell)) * np.sqrt(noise_var)
    ill_nodes = np.zeros(0, dtype=np.int64)
    if dominance is not None:
        # Dense pivot blocks D_a = s_a U diag(sig) V^T (U, V random orthogonal,
        # sig ~ U[1, 2]) with s_a = dominance * sum_b ||A_ab||_F / min(sig):
        # block diagonally dominant by at least `dominance` in the 2-norm.
        # Planted nodes get sig = (1, ..., 1, 1/ill_cond) and s_a =
        # dominance * sum_b ||A_ab||_F, i.e. kappa_2(D_a) = ill_cond exactly.
        u, _ = np.linalg.qr(rng.standard_normal((n_nodes, ell, ell)))
        v, _ = np.linalg.qr(rng.standard_normal((n_nodes, ell, ell)))
        sig = rng.uniform(1.0, 2.0, (n_nodes, ell))
        n_ill = int(round(ill_frac * n_nodes))
        ill_nodes = np.sort(rng.choice(n_nodes, size=n_ill, replace=False)) if n_ill else ill_nodes
        sig[ill_nodes] = 1.0
        sig[ill_nodes, -1] = 1.0 / ill_cond
        z = np.einsum("nij,nj,nkj->nik", u, sig, v)
        if keep is not None:
            keep[diag] = True
        offn = blocks if keep is None else np.where(keep, blocks, 0.0)
        fro = np.sqrt((offn ** 2).sum(axis=(1, 2)))
        fro[diag] = 0.0
        off_sum = np.bincount(row_node, weights=fro, minlength=n_nodes)
        denom = sig.min(axis=1)
        denom[ill_nodes] = 1.0
        s_a = np.where(off_sum > 0, dominance * off_sum / denom, 1.0)
        blocks[diag] = z * s_a[:, None, None]
    m = _expand_blocks(n_nodes, ell, nptr, nidx, blocks, keep)
    m.meta.update(kind="geometric", nodes=n_nodes, ell=ell, seed=seed, radius=r,
                  node_of_row=np.repeat(np.arange(n_nodes), ell), ill_nodes=ill_nodes,
                  approx=approx)
    return _scramble(m, seed + 7919) if scramble else m


def random_sparse(n: int, density: float, seed: int = 0, diag: bool = True,
                  empty_rows: int = 0) -> CSR:
    """Unstructured random pattern with N(0,1) values (edge-case inputs)."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    m = sp.random(n, n, density=density, random_state=rng, format="csr",
                  data_rvs=rng.standard_normal)
    if diag:
        m = m + sp.diags(rng.standard_normal(n) + 4.0 * np.sign(rng.standard_normal(n)))
    m = sp.csr_matrix(m)
    if empty_rows:
        rows = rng.choice(n, size=empty_rows, replace=False)
        m = sp.lil_matrix(m)
        for r in rows:
            m.rows[r] = []
            m.data[r] = []
        m = sp.csr_matrix(m)
    out = _from_scipy(m, dict(kind="random", seed=seed))
    return out


def from_dense(a: np.ndarray, keep_zeros: bool = False) -> CSR:
    """CSR of a dense array (explicit zeros stored when ``keep_zeros``)."""
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[0]
    mask = np.ones_like(a, dtype=bool) if keep_zeros else a != 0
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    rows, cols = np.nonzero(mask)
    return CSR(n, rowptr, cols.astype(np.int32), a[rows, cols].copy(), dict(kind="dense"))


def ones_rhs(m: CSR) -> np.ndarray:
    """b = A * 1, the right-hand side used for every configured workload."""
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    return np.bincount(rows, weights=m.val, minlength=m.n).astype(np.float64)


# Named workloads (sizes and parameters of the configured benchmark cases).
WORKLOADS = {
    "grid10_l5": dict(gen="grid", nx=10, ny=10, nz=10, ell=5, tau=1.0, nlev=2, droptol=1e-3,
                      lfil=20, precision="fp64"),
    "geo60k_l6": dict(gen="geo", n_nodes=60_000, ell=6, tau=0.8, nlev=3, droptol=1e-4,
                      lfil=-1, precision="fp64"),
    "geo500k_l6": dict(gen="geo", n_nodes=500_000, ell=6, tau=0.8, nlev=4, droptol=1e-4,
                       lfil=30, precision="fp32", dominance=1.5, ill_frac=1e-3),
    "geo2m_l6": dict(gen="geo", n_nodes=2_000_000, ell=6, tau=0.9, nlev=5, droptol=1e-5,
                     lfil=40, precision="fp32"),
}


def make_workload(name: str, seed: int = 0, scale: float = 1.0) -> CSR:
    """Build a named workload; ``scale`` shrinks the node count (tests)."""
    w = WORKLOADS[name]
    if w["gen"] == "grid":
        return grid_7pt(w["nx"], w["ny"], w["nz"], w["ell"], seed=seed)
    nn = max(2, int(round(w["n_nodes"] * scale)))
    return geometric(nn, w["ell"], seed=seed, dominance=w.get("dominance"),
                     ill_frac=w.get("ill_frac", 0.0))


# Named batches of independent matrices (batched factorization): count
# matrices from the geometric generator, node counts log-uniform in
# [min_nodes, max_nodes], unknowns per node drawn from ells, matrix k built
# with seed k.
BATCHES = {
    "batch32": dict(count=32, min_nodes=20_000, max_nodes=300_000, ells=(4, 5, 6), tau=0.8, nlev=4,
                    droptol=1e-4, lfil=30, precision="fp32"),
}


def batch_shapes(name: str, seed: int = 0, scale: float = 1.0) -> list[tuple[int, int]]:
    """(nodes, ell) of every matrix of a named batch; ``scale`` shrinks the
    node counts."""
    b = BATCHES[name]
    rng = np.random.default_rng(seed)
    lo, hi = np.log(b["min_nodes"]), np.log(b["max_nodes"])
    nodes = np.exp(rng.uniform(lo, hi, b["count"]))
    ells = rng.choice(np.asarray(b["ells"]), b["count"])
    return [(max(2, int(round(n * scale))), int(e)) for n, e in zip(nodes, ells)]


def make_batch(name: str, seed: int = 0, scale: float = 1.0) -> list[CSR]:
    """The matrices of a named batch (matrix k uses seed ``seed + k``)."""
    return [geometric(n, e, seed=seed + k) for k, (n, e) in enumerate(batch_shapes(name, seed, scale))]
