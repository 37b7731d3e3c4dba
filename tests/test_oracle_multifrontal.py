"""Pins of the multifrontal oracle tier (oracle/multifrontal.py) against independent definitions of
the same answer: a dense LAPACK solve, the SuperLU global direct solve, the residual, invariance to
the dissection (leaf size), and a non-cubic box.  No GPU."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import direct, discretization as disc, multifrontal as mf
from paper_1801_08655_gb300 import workloads as W


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_matches_dense_lapack_solve():
    p = W.small_problem(10, 2, 2, seed=21, R=3)
    f = p.rhs()
    u_mf = mf.solve(p.m, p.omega, p.npml, p.C, f, leaf=27)
    u_dense = direct.solve(p.m, p.omega, p.npml, p.C, f, dense=True)
    assert _rel(u_mf, u_dense) < 1e-12


def test_matches_superlu_and_residual():
    p = W.small_problem(20, 4, 2, seed=22, R=2)
    f = p.rhs()
    u_mf = mf.solve(p.m, p.omega, p.npml, p.C, f, leaf=128)
    u_slu = direct.solve(p.m, p.omega, p.npml, p.C, f)
    assert _rel(u_mf, u_slu) < 1e-11
    A = disc.global_operator(p.m, p.omega, p.npml, p.C)
    S = disc.row_scaling(p.n, p.npml, p.C, p.omega)
    for r in range(p.R):
        b = (S * f[r]).ravel()
        assert np.linalg.norm(A @ u_mf[r].ravel() - b) / np.linalg.norm(b) < 1e-12


def test_independent_of_the_dissection_and_spills_to_disk(tmp_path):
    p = W.small_problem(14, 3, 2, seed=23, R=2)
    f = p.rhs()
    u1 = mf.solve(p.m, p.omega, p.npml, p.C, f, leaf=8)
    u2 = mf.solve(p.m, p.omega, p.npml, p.C, f, leaf=400, spill_dir=str(tmp_path))
    assert _rel(u1, u2) < 1e-12
    assert not any(tmp_path.iterdir()) or all(not any(d.iterdir()) for d in tmp_path.iterdir())


def test_non_cubic_box_against_dense():
    rng = np.random.default_rng(5)
    nz, ny, nx = 7, 9, 11
    m = 0.5 + rng.random((nz, ny, nx))
    omega = 1.1

    def prof(n):
        sn = 1.0 + 1j * rng.random(n) * 0.3
        sh = 1.0 + 1j * rng.random(n + 1) * 0.3
        return sn, sh

    A = disc.assemble(m, omega, prof(nx), prof(ny), prof(nz))
    B = rng.standard_normal((nz * ny * nx, 3)) + 1j * rng.standard_normal((nz * ny * nx, 3))
    x = mf.MultifrontalSolver(A, (nz, ny, nx), leaf=20).solve(B)
    x_ref = sla.solve(A.toarray(), B)
    assert _rel(x, x_ref) < 1e-12
    # a single right-hand side as a vector
    x1 = mf.MultifrontalSolver(A, (nz, ny, nx), leaf=20).solve(B[:, 0])
    assert x1.shape == (nz * ny * nx,) and _rel(x1, x_ref[:, 0]) < 1e-12


def test_symbolic_rejects_a_tree_that_does_not_separate():
    A = disc.assemble(np.ones((4, 4, 6)), 1.0, *[disc.global_profiles(k, 0, 0.0, 1.0) for k in (6, 4, 4)])
    nodes = mf.dissection_tree(4, 4, 6, leaf=16)
    # swap the own sets of the two leaves under the root's first child: a leaf then owns cells
    # coupled to cells of its sibling that are eliminated later, which the check must reject
    leaves = [k for k, nd in enumerate(nodes) if not nd.children]
    a, b = leaves[0], leaves[-1]
    nodes[a].own, nodes[b].own = nodes[b].own.copy(), nodes[a].own.copy()
    e = 0
    for nd in nodes:
        nd.s, nd.t = e, e + nd.own.size
        e = nd.t
    perm = np.concatenate([nd.own for nd in nodes])
    Ap = A.tocsr()[perm][:, perm].tocsr()
    Ap.sort_indices()
    with pytest.raises(ValueError):
        mf.symbolic(nodes, Ap)


def test_stored_128cube_reference_is_consistent():
    """The stored 128^3 oracle values (tests/golden/make_golden_cfg3.py) belong to the 128^3
    workload's sources, come from a solve whose residual is at rounding level, and are
    self-consistent (samples bounded by the full norms, physical-region norms below the full ones,
    sketches of the right magnitude: E|<w, u>|^2 = ||u||^2)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cfg3_128cube_layered_block.npz")
    ref = np.load(path)
    p = W.config(3)
    assert np.array_equal(ref["sources"], p.sources)
    assert ref["u"].shape == (p.R, ref["idx"].size) and ref["sketch"].shape == (p.R, int(ref["sketch_k"]))
    assert np.all(ref["relres"] < 1e-12)
    assert np.all(np.linalg.norm(ref["u"], axis=1) < ref["norms"])
    assert np.all(ref["norms_phys"] < ref["norms"])
    ratio = np.sqrt(np.mean(np.abs(ref["sketch"]) ** 2, axis=1)) / ref["norms"]
    assert np.all((ratio > 0.4) & (ratio < 2.0)), ratio.min()
