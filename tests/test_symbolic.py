"""The library's symbolic phase (hz_symbolic_shape: the geometric nested dissection hz_create runs
for every slab shape) against the oracle's generic multifrontal symbolic phase, bit for bit, on
the CPU.  The library's tree (own unknowns, parents, elimination order) is handed to the oracle,
which derives every update set from the graph of the 7-point operator alone (couplings of a
node's own unknowns plus its children's update sets, minus its own) and checks that the tree is
an assembly tree; the library's update sets, built from the geometry (the face shell of each
subtree box), must be exactly those.  Integer work: compared for equality."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import multifrontal as mf
from paper_1801_08655_gb300 import build, hz


def seven_point_pattern(nz, ny, nx):
    """Sparsity pattern of a 7-point operator on an (nz, ny, nx) box, x fastest."""
    def path(n):
        return sp.diags([np.ones(n - 1), np.ones(n), np.ones(n - 1)], [-1, 0, 1], format="csr")
    Ix, Iy, Iz = (sp.identity(n, format="csr") for n in (nx, ny, nz))
    A = (sp.kron(sp.kron(Iz, Iy), path(nx)) + sp.kron(sp.kron(Iz, path(ny)), Ix)
         + sp.kron(sp.kron(path(nz), Iy), Ix)).tocsr()
    A.eliminate_zeros()     # the pattern: stored entries only where the stencil couples
    assert A.nnz == 7 * nx * ny * nz - 2 * (ny * nz + nx * nz + nx * ny)
    return A


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


@pytest.mark.parametrize("nx,ny,nz,leaf", [(5, 5, 5, 8), (8, 8, 12, 16), (10, 7, 9, 32), (16, 16, 22, 256),
                                           (24, 24, 17, 256), (20, 20, 27, 64), (12, 9, 26, 1)])
def test_update_sets_match_the_generic_symbolic_phase(nx, ny, nz, leaf):
    d = hz.symbolic_shape(nx, ny, nz, leaf)
    N = nx * ny * nz
    perm = d["perm"].astype(np.int64)
    assert np.array_equal(np.sort(perm), np.arange(N))               # a permutation of the cells
    n_nodes = d["own0"].size
    # post-order: node k's own unknowns follow those of all its descendants, contiguously
    assert d["own0"][0] == 0 and np.all(d["own0"][1:] == d["own0"][:-1] + d["nown"][:-1])
    assert d["own0"][-1] + d["nown"][-1] == N and d["parent"][-1] == -1
    assert np.all(d["parent"][:-1] > np.arange(n_nodes - 1))
    nodes = []
    for k in range(n_nodes):
        s0, n = int(d["own0"][k]), int(d["nown"][k])
        kids = [int(c) for c in np.nonzero(d["parent"] == k)[0]]
        nodes.append(mf.TreeNode(own=perm[s0:s0 + n], children=kids, s=s0, t=s0 + n))
    A = seven_point_pattern(nz, ny, nx)
    Ap = A[perm][:, perm].tocsr()
    Ap.sort_indices()
    mf.symbolic(nodes, Ap)                                            # raises unless an assembly tree
    ends = np.append(d["upd_off"][1:], d["upd_idx"].size)
    for k, nd in enumerate(nodes):
        lib_upd = d["upd_idx"][d["upd_off"][k]:ends[k]]
        assert np.array_equal(lib_upd, nd.upd), (k, lib_upd[:8], nd.upd[:8])


def test_bad_sizes_are_statuses():
    with pytest.raises(hz.HzError) as e:
        hz.symbolic_shape(0, 4, 4, 8)
    assert e.value.status == hz.HZ_ERR_ARG
    with pytest.raises(hz.HzError) as e:
        hz.symbolic_shape(4, 4, 4, 0)
    assert e.value.status == hz.HZ_ERR_ARG
