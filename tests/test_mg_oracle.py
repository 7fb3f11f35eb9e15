"""Pins of the multigrid V-cycle reference (oracle/mg_oracle.py), CPU only.

Each pin comes from outside the reference itself: the published SplitMix64
output sequence, closed forms of linear interpolation and of the Galerkin
product of the 1D Laplacian, the exact inverse on a one-level hierarchy, the
spectrum of the 2D Laplacian, and the textbook contraction of a multigrid
V-cycle on the Poisson problem.
"""
import numpy as np
import scipy.sparse as sp

from oracle import mg_oracle as G


def _laplacian(dims, fixed_nodes):
    """Unscaled 5-point (2D) or 3-point (1D) Laplacian over the nodes of a
    grid, prescribed nodes replaced by identity rows and columns."""
    mats = []
    for n in dims:
        mats.append(sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]))
    A = mats[0]
    for k, m in enumerate(mats[1:], start=1):
        A = sp.kron(sp.eye(dims[k]), A) + sp.kron(m, sp.eye(int(np.prod(dims[:k]))))
    keep = ~fixed_nodes
    K = sp.diags(keep.astype(float))
    return (K @ A @ K + sp.diags(fixed_nodes.astype(float))).tocsr()


def _boundary(dims):
    idx = np.indices(dims[::-1]).reshape(len(dims), -1)[::-1]   # x fastest
    b = np.zeros(idx.shape[1], dtype=bool)
    for a, n in enumerate(dims):
        b |= (idx[a] == 0) | (idx[a] == n - 1)
    return b


def test_splitmix64_published_sequence():
    """SplitMix64 seeded with 1234567 (states advanced by the gamma) gives
    the sequence of the reference implementation; seed 0 gives
    0xE220A8397B1DCDAF."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    s = 1234567
    got = []
    for _ in range(5):
        got.append(G.splitmix64(s))
        s = (s + G.GAMMA) & ((1 << 64) - 1)
    assert got == want
    assert G.splitmix64(0) == 0xE220A8397B1DCDAF
    u = G.splitmix_unit(np.arange(20000))
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.02


def test_prolongation_exact_for_linear_fields():
    """Linear interpolation reproduces a linear field at every fine node;
    rows of DOFs not kept are zero."""
    fd, cd, B = [9, 7], [5, 4], 2
    X, Y = np.meshgrid(np.arange(cd[0]), np.arange(cd[1]), indexing="xy")
    coarse = np.stack([2.0 * X.ravel() + 3.0 * Y.ravel(), -X.ravel() + 0.5 * Y.ravel()], axis=1).ravel()
    keep = np.ones(np.prod(fd) * B, dtype=bool)
    keep[5] = False
    P = G.prolongation(fd, cd, B, keep)
    x, y = np.meshgrid(np.arange(fd[0]) / 2.0, np.arange(fd[1]) / 2.0, indexing="xy")
    fine = np.stack([2.0 * x.ravel() + 3.0 * y.ravel(), -x.ravel() + 0.5 * y.ravel()], axis=1).ravel()
    got = P @ coarse
    assert np.allclose(got[keep], fine[keep], rtol=0, atol=1e-13)
    assert got[5] == 0.0


def test_galerkin_of_1d_laplacian():
    """P^T A P of the 1D Laplacian [-1 2 -1] with linear interpolation is
    half the coarse Laplacian in the interior."""
    n = 65
    fixed = np.zeros(n, dtype=bool)
    fixed[[0, n - 1]] = True
    A = _laplacian([n], fixed)
    H = G.Hierarchy(A, np.ones(n, dtype=bool), fixed, [n], 1, dense_max=16)
    Ac = H.A[1].toarray()
    nc = H.dims[1][0]
    assert nc == 33
    for i in range(2, nc - 2):
        assert np.allclose(Ac[i, i - 1:i + 2], [-0.5, 1.0, -0.5], rtol=0, atol=1e-14), i
    # the coarse end nodes interpolate to the free fine nodes 1 and n-2, so
    # they are not prescribed; the product of a symmetric A stays symmetric
    assert not H.fix[1].any()
    assert np.allclose(Ac, Ac.T, rtol=0, atol=1e-14)


def test_single_level_hierarchy_is_the_exact_inverse():
    dims = [8, 7]
    fixed = _boundary(dims)
    fixed[:] = False
    fixed[[0, 1]] = True
    A = _laplacian(dims, fixed) + sp.eye(np.prod(dims)) * 0.1
    H = G.Hierarchy(A, np.ones(np.prod(dims), dtype=bool), fixed, dims, 1, dense_max=128)
    assert H.L == 1
    b = np.random.default_rng(3).standard_normal(np.prod(dims))
    z = H.vcycle(b)
    assert np.allclose(z, np.linalg.solve(A.toarray(), b), rtol=0, atol=1e-12)


def test_power_estimate_of_laplacian():
    """D^-1 A of the 2D Laplacian with Dirichlet nodes eliminated is A/4,
    whose largest eigenvalue is 1 + cos(pi/(n-1)) over the interior; eight
    power iterations from the fixed start vector approach it from below."""
    n = 33
    dims = [n, n]
    fixed = _boundary(dims)
    A = _laplacian(dims, fixed)
    act = np.ones(n * n, dtype=bool)
    Dinv = np.array([[[1.0 / A[k, k]]] for k in range(n * n)])
    lam = G.power_lambda(A, Dinv, act, fixed, 1, 8)
    free = ~fixed
    Af = A[free][:, free].toarray() / 4.0
    rho = float(np.max(np.linalg.eigvalsh(Af)))
    assert abs(rho - (1.0 + np.cos(np.pi / (n - 1)))) < 1e-12
    assert lam <= rho * (1 + 1e-12) and lam >= 0.8 * rho, (lam, rho)


def test_vcycle_contracts_on_poisson():
    """As a stationary iteration x <- x + M (b - A x) the V-cycle reduces the
    error of the 2D Poisson problem by a factor well below 1 per cycle,
    independently of the grid size (the property multigrid is built for)."""
    factors = []
    for n in (33, 65):
        dims = [n, n]
        fixed = _boundary(dims)
        A = _laplacian(dims, fixed)
        H = G.Hierarchy(A, np.ones(n * n, dtype=bool), fixed, dims, 1)
        assert H.L >= 3
        rng = np.random.default_rng(7)
        xs = np.where(fixed, 0.0, rng.standard_normal(n * n))
        b = A @ xs
        x = np.zeros(n * n)
        errs = []
        for _ in range(8):
            x = x + H.vcycle(b - A @ x)
            errs.append(np.linalg.norm(x - xs))
        rate = (errs[-1] / errs[2]) ** (1.0 / 5)
        factors.append(rate)
        assert rate < 0.35, (n, rate)
    assert abs(factors[0] - factors[1]) < 0.15, factors


def test_block_vcycle_of_decoupled_components():
    """Two uncoupled copies of the 2D Laplacian as one operator with 2x2 node
    blocks (component fastest): the block V-cycle is the scalar V-cycle of
    each component, which pins the node-block indexing of the smoother,
    and the prolongation per component."""
    n = 33
    dims = [n, n]
    fixed1 = _boundary(dims)
    A1 = _laplacian(dims, fixed1)
    A2 = sp.kron(A1, sp.eye(2)).tocsr()
    fixed2 = np.repeat(fixed1, 2)
    act = np.ones(n * n, dtype=bool)
    H1 = G.Hierarchy(A1, act, fixed1, dims, 1)
    rng = np.random.default_rng(11)
    b1 = np.where(fixed1, 0.0, rng.standard_normal(n * n))
    b2 = np.zeros(2 * n * n)
    b2[0::2] = b1
    # the same depth (twice the unknowns per node, twice the dense bound) and
    # the same damping on both sides: the block hierarchy's estimate comes
    # from a different start vector, so its smoother takes H1's damping
    H2c = G.Hierarchy(A2, act, fixed2, dims, 2, dense_max=2 * (H1.act[-1].sum()))
    assert H2c.L == H1.L
    for l in range(H1.L - 1):
        w1 = 1.2 / H1.lam[l] if 1e-3 <= H1.lam[l] < 1e30 else 0.5
        w2 = 1.2 / H2c.lam[l] if 1e-3 <= H2c.lam[l] < 1e30 else 0.5
        H2c.Dinv[l] = H2c.Dinv[l] * (w1 / w2)
    z2 = H2c.vcycle(b2)
    z1 = H1.vcycle(b1)
    assert np.allclose(z2[0::2], z1, rtol=0, atol=1e-12 * np.abs(z1).max())
    assert np.all(z2[1::2] == 0.0)
