"""The seeded input generators: reproducible, and drawing what the recipes say.

Both the oracle and the CUDA path are fed from these generators, so a recipe
that silently changed (another distribution, another seed stream) would shift
every parity case and bench line at once.  These tests pin the recipes: fixed
seeds give identical arrays, the shapes and dtypes are the library's input
format, and the distributions have the properties their docstrings state.
"""
import numpy as np
import pytest

from paper_2210_12859_gb300 import synth


def test_uniform_is_reproducible_and_bounded():
    a = synth.uniform(4096, 3, -0.1, 1.1, seed=7)
    b = synth.uniform(4096, 3, -0.1, 1.1, seed=7)
    c = synth.uniform(4096, 3, -0.1, 1.1, seed=8)
    assert a.dtype == np.float32 and a.shape == (4096, 3)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    assert a.min() >= np.float32(-0.1) and a.max() <= np.float32(1.1)
    # uniform: mean near the box centre, variance near (hi - lo)^2 / 12
    assert abs(float(a.mean()) - 0.5) < 0.02
    assert abs(float(a.var()) - 1.2 ** 2 / 12.0) < 0.01


def test_uniform_small_recipe():
    pts, qs = synth.uniform_small(2048, 1024)
    assert pts.shape == (2048, 3) and qs.shape == (1024, 3)
    assert pts.min() >= 0.0 and pts.max() <= 1.0
    assert qs.min() >= np.float32(-0.1) and qs.max() <= np.float32(1.1)
    # queries reach outside the data box, so some lie outside [0,1]^3
    assert np.any((qs < 0.0) | (qs > 1.0))
    pts2, qs2 = synth.uniform_small(2048, 1024)
    assert np.array_equal(pts, pts2) and np.array_equal(qs, qs2)


def test_gmm_sample_clusters_around_centres():
    mix = synth.gmm_mixture(16, 3, 0.01, seed=3)
    assert mix.centres.shape == (16, 3) and np.all(mix.sigmas == 0.01)
    pts = synth.gmm_sample(mix, 20000, seed=4)
    assert pts.dtype == np.float32 and pts.shape == (20000, 3)
    d = np.linalg.norm(pts[:, None, :].astype(np.float64) - mix.centres[None], axis=2).min(axis=1)
    # the distance to the own centre is sigma * chi_3; P(chi_3 > 6) is below
    # 1e-7, so no mixture point is farther than 6 sigma from every centre
    assert d.max() < 6 * 0.01
    # and the median of sigma * chi_3 is about 1.54 sigma (the nearest
    # centre can only be closer, never farther)
    assert np.median(d) < 1.6 * 0.01


def test_gmm_queries_uniform_share():
    mix = synth.gmm_mixture(8, 3, 0.005, seed=5)
    q = synth.gmm_queries(mix, 50000, 0.1, seed=6)
    assert q.dtype == np.float32 and q.shape == (50000, 3)
    d = np.linalg.norm(q[:, None, :].astype(np.float64) - mix.centres[None], axis=2).min(axis=1)
    far = d > 6 * 0.005
    # mixture draws never land this far out; a uniform draw lands within 6
    # sigma of one of 8 centres with probability at most 8 * 4/3 pi (0.03)^3,
    # about 1e-3, so the far share estimates the uniform share
    assert abs(far.mean() - 0.1) < 0.01
    assert np.all(q[far] >= 0.0) and np.all(q[far] <= 1.0)
    assert np.array_equal(q, synth.gmm_queries(mix, 50000, 0.1, seed=6))


def test_gmm_query_is_uniform_marks_the_uniform_draws():
    """The mask of uniformly drawn queries: those lie in the cube and (but for
    the ~1e-3 that land near a centre) farther than 6 sigma from every centre,
    the others within it."""
    mix = synth.gmm_mixture(8, 3, 0.005, seed=5)
    q = synth.gmm_queries(mix, 50000, 0.1, seed=6)
    uni = synth.gmm_query_is_uniform(50000, 0.1, seed=6)
    d = np.linalg.norm(q[:, None, :].astype(np.float64) - mix.centres[None], axis=2).min(axis=1)
    assert np.all(d[~uni] < 6 * 0.005)
    assert np.mean(d[uni] > 6 * 0.005) > 0.99
    assert np.all(q[uni] >= 0.0) and np.all(q[uni] <= 1.0)
    assert abs(uni.mean() - 0.1) < 0.005


def test_gmm_queries_without_uniform_share():
    mix = synth.gmm_mixture(8, 3, 0.005, seed=5)
    q = synth.gmm_queries(mix, 20000, 0.0, seed=6)
    d = np.linalg.norm(q[:, None, :].astype(np.float64) - mix.centres[None], axis=2).min(axis=1)
    assert d.max() < 6 * 0.005


def test_gmm_large_recipe_small_size():
    pts, qs = synth.gmm_large(4096, 4096)
    assert pts.shape == (4096, 3) and qs.shape == (4096, 3)
    assert pts.dtype == np.float32 and qs.dtype == np.float32
    mix = synth.gmm_mixture(64, 3, 0.01, synth.BASE_SEED + 2)
    d = np.linalg.norm(pts[:, None, :].astype(np.float64) - mix.centres[None], axis=2).min(axis=1)
    assert d.max() < 6 * 0.01
    # points and queries are separate draws
    assert not np.array_equal(pts, qs)


def test_surface_points_lie_on_their_shapes():
    sh = synth.surface_shapes(32, seed=11)
    assert sh.centre.shape == (32, 3) and sh.axis.shape == (32, 3)
    assert np.allclose(np.linalg.norm(sh.axis, axis=1), 1.0)
    assert np.all((sh.R >= 0.01) & (sh.R <= 0.1))
    assert np.all(sh.r < sh.R)
    pts = synth.surface_sample(sh, 20000, seed=12, jitter=0.0).astype(np.float64)
    assert pts.shape == (20000, 3)
    # the implicit distance of each point to the nearest shape surface:
    # sphere |x - c| - R, torus sqrt((rho - R)^2 + h^2) - r with h the
    # height along the axis and rho the distance from the axis
    best = np.full(len(pts), np.inf)
    for s in range(32):
        v = pts - sh.centre[s]
        if sh.kind[s] == 0:
            f = np.abs(np.linalg.norm(v, axis=1) - sh.R[s])
        else:
            h = v @ sh.axis[s]
            rho = np.sqrt(np.maximum((v * v).sum(axis=1) - h * h, 0.0))
            f = np.abs(np.sqrt((rho - sh.R[s]) ** 2 + h * h) - sh.r[s])
        best = np.minimum(best, f)
    # float32 storage of coordinates near 1 rounds by about 6e-8
    assert best.max() < 1e-6


def test_surface_torus_sampling_is_area_uniform():
    # one torus: with area-uniform sampling the minor angle v has density
    # proportional to R + r cos v, so E[cos v] = r / (2 R)
    sh = synth.surface_shapes(1, seed=0)
    sh.kind[:] = 1
    sh.centre[:] = 0.5
    sh.R[:] = 0.1
    sh.r[:] = 0.05
    sh.axis[:] = np.array([0.0, 0.0, 1.0])
    sh.area[:] = 4 * np.pi ** 2 * 0.1 * 0.05
    pts = synth.surface_sample(sh, 200000, seed=1, jitter=0.0).astype(np.float64)
    v = pts - 0.5
    rho = np.sqrt(v[:, 0] ** 2 + v[:, 1] ** 2)
    cos_v = (rho - 0.1) / 0.05
    assert abs(cos_v.mean() - 0.05 / (2 * 0.1)) < 0.01
    # a plain uniform minor angle would give E[cos v] = 0
    assert cos_v.mean() > 0.2


def test_surface_set_reproducible():
    a = synth.surface_set(1000, 500)
    b = synth.surface_set(1000, 500)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0][:500], a[1])


def test_clouds_sizes_and_offsets():
    c = synth.clouds(64, 8.0, 12.0, seed=9)
    sizes = np.diff(c.offsets)
    assert len(c.offsets) == 65 and c.offsets[0] == 0
    assert np.all(sizes >= 2 ** 8) and np.all(sizes <= 2 ** 12)
    assert c.points.shape == (int(c.offsets[-1]), 3) and c.points.dtype == np.float32
    assert np.array_equal(c.offsets, c.qoffsets) and c.queries.shape == c.points.shape
    # log-uniform sizes: the mean of log2 N_i is near the middle of the range
    assert abs(float(np.log2(sizes).mean()) - 10.0) < 0.5
    d = synth.clouds(64, 8.0, 12.0, seed=9)
    assert np.array_equal(c.points, d.points) and np.array_equal(c.queries, d.queries)


@pytest.mark.parametrize("D", [2, 4, 8])
def test_uniform_dim(D):
    pts, qs = synth.uniform_dim(1000, 500, D)
    assert pts.shape == (1000, D) and qs.shape == (500, D)
    assert pts.min() >= 0.0 and pts.max() <= 1.0
    assert not np.array_equal(pts[:500], qs)
