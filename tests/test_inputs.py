"""The seeded workload generators produce what their recipe states: rigid
waters (O-H 0.96 A, H-O-H 104.5 deg) on a jittered 3.0 A grid with no close
contacts, 25 Cartesian functions per water, reproducible streams."""
import numpy as np
import pytest

from paper_1708_00033_gb300 import inputs as I

A = I.ANGSTROM_IN_BOHR


@pytest.mark.parametrize("n,cfg,idx", [(1, 1, 0), (4, 1, 0), (16, 2, 3), (64, 2, 0)])
def test_water_geometry_recipe(n, cfg, idx):
    g = I.water_cluster(n, cfg, idx)
    assert g.n_atoms == 3 * n
    Z = g.Z.reshape(n, 3)
    assert np.all(Z[:, 0] == 8) and np.all(Z[:, 1:] == 1)
    x = g.xyz.reshape(n, 3, 3) / A  # angstrom
    oh1 = np.linalg.norm(x[:, 1] - x[:, 0], axis=1)
    oh2 = np.linalg.norm(x[:, 2] - x[:, 0], axis=1)
    assert np.allclose(oh1, 0.96, atol=1e-12) and np.allclose(oh2, 0.96, atol=1e-12)
    cos = np.einsum("ij,ij->i", x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]) / (oh1 * oh2)
    assert np.allclose(np.degrees(np.arccos(cos)), 104.5, atol=1e-9)
    # oxygen on its grid point within the jitter
    m = int(np.ceil(n ** (1.0 / 3.0) - 1e-9))
    for k in range(n):
        grid = 3.0 * np.array([k % m, (k // m) % m, k // (m * m)], dtype=float)
        assert np.all(np.abs(x[k, 0] - grid) <= 0.3 + 1e-12)
    # no intermolecular contact below 1.6 A
    for a in range(n):
        for b in range(a):
            d = np.linalg.norm(x[a][:, None, :] - x[b][None, :, :], axis=2)
            assert d.min() >= 1.6


def test_streams_are_reproducible_and_distinct():
    a = I.water_cluster(8, 2, 5)
    b = I.water_cluster(8, 2, 5)
    c = I.water_cluster(8, 2, 6)
    d = I.water_cluster(8, 3, 5)
    assert np.array_equal(a.xyz, b.xyz)
    assert not np.allclose(a.xyz, c.xyz) and not np.allclose(a.xyz, d.xyz)
    G1 = I.random_orbitals(50, 10, 1, 0)
    assert np.array_equal(G1, I.random_orbitals(50, 10, 1, 0))
    assert not np.allclose(G1, I.random_orbitals(50, 10, 1, 1))


def test_subset_is_prefix_of_the_cluster():
    g = I.water_cluster(256, I.CONFIG_MIXED, 0)
    s = I.subset_waters(g, 16)
    assert np.array_equal(s.xyz, g.xyz[: 48]) and np.array_equal(s.Z, g.Z[: 48])


@pytest.mark.parametrize("n", [1, 4, 64])
def test_basis_counts(n):
    g = I.water_cluster(n, 2, 0)
    b = I.synthetic_basis(g)
    assert b.n_shells == 12 * n and b.n_bf == 25 * n
    assert np.all(b.nprim == 3)
    assert I.n_electrons(g) == 10 * n
    # exponents alpha * {1, 3, 9}, coefficients {0.4, 0.4, 0.2}, shells in the element's order
    off = b.prim_offsets()
    for s in range(12):
        e = b.exps[off[s]:off[s + 1]]
        assert np.allclose(e / e[0], [1.0, 3.0, 9.0])
        assert np.allclose(b.coefs[off[s]:off[s + 1]], [0.4, 0.4, 0.2])
    assert list(b.l[:12]) == [0, 0, 0, 1, 1, 2, 0, 0, 1, 0, 0, 1]


def test_batch_sizes_in_range():
    sizes = I.batch_cluster_sizes(512)
    assert len(sizes) == 512 and min(sizes) >= 1 and max(sizes) <= 16
    assert len(set(sizes)) > 10
