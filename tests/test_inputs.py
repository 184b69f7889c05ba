"""The seeded synthetic inputs (paper_2108_07031_gb300/cloud.py): the cloud
recipe that stands in for the paper's NACA 0012 point distributions, the
shuffled order, ragged packing and the condition sets. CPU only."""

import numpy as np
import pytest

from paper_2108_07031_gb300 import cloud as Cl


@pytest.fixture(scope="module")
def small():
    return Cl.naca0012_cloud(64, 20)


def test_generator_is_deterministic(small):
    again = Cl.naca0012_cloud(64, 20)
    for f in ("xy", "normals", "flags", "nbr_offsets", "nbr_idx"):
        assert np.array_equal(getattr(small, f), getattr(again, f)), f


def test_flags_normals_and_stencils_are_valid(small):
    n_c = small.n_c
    assert np.all(small.flags[:n_c] == 1)                 # wall loop first
    assert np.count_nonzero(small.flags == 1) == n_c
    assert np.count_nonzero(small.flags == 2) == n_c      # one far-field layer
    bnd = small.flags != 0
    assert np.allclose(np.hypot(small.normals[bnd, 0], small.normals[bnd, 1]), 1.0)
    # wall normals point into the fluid (away from the airfoil's centre)
    cx = small.xy[:n_c].mean(0)
    assert np.all(((small.xy[:n_c] - cx) * small.normals[:n_c]).sum(1) > 0)
    cnt = np.diff(small.nbr_offsets)
    assert cnt.min() >= 3 and cnt.max() <= Cl.MAX_NEIGHBOURS
    for i in range(small.n):
        nb = small.neighbours(i)
        assert i not in nb and len(set(nb.tolist())) == len(nb)
        assert nb.min() >= 0 and nb.max() < small.n


def test_wall_follows_the_naca0012_thickness(small):
    x, y = small.xy[:small.n_c, 0], small.xy[:small.n_c, 1]
    assert np.allclose(np.abs(y), Cl.naca0012_half_thickness(x), atol=1e-12)
    assert x.min() >= 0.0 and x.max() <= 1.0 + 1e-12


def test_far_field_is_a_circle_of_twenty_chords(small):
    far = small.xy[small.flags == 2]
    r = np.hypot(far[:, 0] - 0.5, far[:, 1])
    assert np.allclose(r, 20.0, rtol=1e-12)


def test_shuffled_cloud_is_a_relabelling(small):
    sh = Cl.naca0012_cloud(64, 20, shuffle=True)
    assert np.array_equal(sh.xy[:sh.n_c], small.xy[:small.n_c])  # wall points stay first
    key = lambda xy: np.lexsort((xy[:, 1], xy[:, 0]))  # noqa: E731
    assert np.array_equal(sh.xy[key(sh.xy)], small.xy[key(small.xy)])
    # the same stencils up to the relabelling
    order = np.empty(sh.n, dtype=np.int64)
    order[key(sh.xy)] = key(small.xy)  # shuffled index -> unshuffled index
    for i in range(0, sh.n, 37):
        a = np.sort(order[sh.neighbours(i)])
        b = np.sort(small.neighbours(order[i]))
        assert np.array_equal(a, b)


def test_cloud_dims_of_the_benchmark_sizes():
    assert Cl.cloud_dims(5_120) == (128, 40)
    assert Cl.cloud_dims(600_000) == (1386, 433)
    assert Cl.cloud_dims(2_500_000) == (2828, 884)
    assert Cl.cloud_dims(10_000_000) == (5658, 1768)


def test_pack_offsets_and_shifted_connectivity():
    a, b = Cl.naca0012_cloud(24, 8), Cl.naca0012_cloud(32, 10, seed=3)
    p, offs = Cl.pack([a, b])
    assert list(offs) == [0, a.n, a.n + b.n]
    assert np.array_equal(p.xy[a.n:], b.xy)
    for i in (0, 5, b.n - 1):
        assert np.array_equal(p.neighbours(a.n + i), b.neighbours(i) + a.n)
        assert np.array_equal(p.neighbours(i % a.n), a.neighbours(i % a.n))


def test_condition_and_ragged_size_sets():
    m, al = Cl.conditions(64)
    assert m.min() >= 0.3 and m.max() <= 0.8 and al.min() >= -4.0 and al.max() <= 6.0
    m2, al2 = Cl.conditions(64)
    assert np.array_equal(m, m2) and np.array_equal(al, al2)
    sizes = Cl.ragged_sizes(16)
    assert len(sizes) == 16 and min(sizes) >= 100_000 and max(sizes) <= 1_000_000
    assert sizes == Cl.ragged_sizes(16)
