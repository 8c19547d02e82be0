"""The seeded input generator against the recipe it states (module docstring
of synth.py): STFT bins, geometries, direction grids, free-field steering,
the noise field's spectrum, source power, shapes, dtypes and determinism.
CPU only; the generator holds none of the method's arithmetic."""

import numpy as np
import pytest

from paper_2504_03373_gb300 import synth


def test_bin_frequencies():
    f = synth.bin_frequencies()
    assert f.shape == (209,)
    assert f[0] == 500.0 and f[-1] == 7000.0  # k = 16 and k = 224 at 31.25 Hz per bin
    assert np.allclose(np.diff(f), 31.25)


def test_direction_grids():
    g = synth.sphere_grid()
    assert (g.n_az, g.n_el, g.D) == (72, 19, 1368)
    u = g.unit_vectors()
    assert u.shape == (1368, 3)
    assert np.allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-15)
    # flat index d = el_idx * n_az + az_idx; the pole rows are single points
    assert np.array_equal(u[:72], np.tile([0.0, 0.0, -1.0], (72, 1)))
    assert np.array_equal(u[-72:], np.tile([0.0, 0.0, 1.0], (72, 1)))
    a = synth.azimuth_grid()
    assert (a.n_az, a.n_el) == (72, 1)
    assert np.array_equal(a.unit_vectors()[18], [0.0, 1.0, 0.0])  # azimuth 90 deg


def test_array_geometries():
    p = synth.uca(8, 0.1)
    assert np.allclose(np.linalg.norm(p, axis=1), 0.1)
    assert np.all(p[:, 2] == 0.0)
    ang = np.mod(np.arctan2(p[:, 1], p[:, 0]), 2 * np.pi)
    assert np.allclose(ang, 2 * np.pi * np.arange(8) / 8)
    q = synth.ball(2000, 0.4, np.random.default_rng(0))
    r = np.linalg.norm(q, axis=1)
    assert r.max() <= 0.4
    # uniform in the ball: P(r < R/2) = 1/8
    assert abs(np.mean(r < 0.2) - 0.125) < 0.03


def test_free_field_steering():
    rng = np.random.default_rng(1)
    pos = synth.ball(5, 0.4, rng)
    pos[0] = 0.0  # a microphone at the origin sees no delay
    u = synth.sphere_grid().unit_vectors()[::97]
    f = synth.bin_frequencies()
    H = synth.steering(pos, u, f)
    assert H.shape == (209, u.shape[0], 5)
    assert np.allclose(np.abs(H), 1.0)
    assert np.allclose(H[..., 0], 1.0)
    # the opposite direction gives the conjugate response
    assert np.allclose(synth.steering(pos, -u, f), np.conj(H))


def test_noise_field_spectrum_and_unitarity():
    rng = np.random.default_rng(3)
    Q = synth.haar_unitary(rng, 4, 12)
    assert np.allclose(np.matmul(np.conj(np.swapaxes(Q, 1, 2)), Q), np.eye(12), atol=1e-12)
    G = synth.noise_mixing(rng, 4, 12, 1e3)
    K = np.matmul(G, np.conj(np.swapaxes(G, 1, 2)))
    lam = np.linalg.eigvalsh(K)[:, ::-1]
    assert np.allclose(lam, np.logspace(0, -3, 12)[None, :], rtol=1e-9)


@pytest.fixture(scope="module")
def uca8():
    return synth.uca8_single_source(seed=5, nblk=2)


def test_uca8_workload(uca8):
    w = uca8
    assert w.X.shape == (2, 50, 209, 8) and w.X.dtype == np.complex64
    assert w.Xnoise.shape == (50, 209, 8) and w.Xnoise.dtype == np.complex64
    assert w.H.shape == (209, 72, 8)
    assert w.K_true.shape == (209, 8, 8)
    assert (w.Ns, w.T, w.nblk, w.B, w.M, w.D) == (1, 50, 2, 209, 8, 72)
    # the source sits on the grid, at the grid's own direction
    d = int(w.src_grid_idx[0, 0])
    assert 0 <= d < 72
    assert np.allclose(w.src_dirs[0, 0], w.grid.unit_vectors()[d])
    # 0 dB: the source adds as much power per channel as the noise has
    noise = np.mean(np.real(np.einsum("bii->b", w.K_true))) / 8
    assert abs(np.mean(np.abs(w.Xnoise) ** 2) / noise - 1.0) < 0.05
    assert abs(np.mean(np.abs(w.X) ** 2) / noise - 2.0) < 0.1


def test_ball60_workload_shape_and_recipe():
    w = synth.ball60_three_sources(seed=2, nblk=1)
    assert w.X.shape == (1, 50, 209, 60)
    assert w.Xnoise.shape == (240, 209, 60)
    assert w.H.shape == (209, 1368, 60)
    assert np.linalg.norm(w.pos, axis=1).max() <= 0.4
    assert w.snr_db.shape == (3,) and np.all((w.snr_db >= -5.0) & (w.snr_db <= 10.0))
    assert np.all(w.src_grid_idx == -1)  # continuous directions
    assert np.allclose(np.linalg.norm(w.src_dirs, axis=-1), 1.0)
    lam = np.linalg.eigvalsh(w.K_true[::50])
    assert np.allclose(lam.max(1) / lam.min(1), 1e3, rtol=1e-6)


def test_seeded_and_deterministic():
    a = synth.uca8_single_source(seed=9)
    b = synth.uca8_single_source(seed=9)
    c = synth.uca8_single_source(seed=10)
    for name in ("X", "Xnoise", "K_true", "H"):
        assert np.array_equal(getattr(a, name), getattr(b, name))
    assert not np.array_equal(a.X, c.X)


def test_drift_moves_sources_in_azimuth():
    w = synth.make_workload(M=8, T=10, nblk=3, Ns=1, geometry="uca", radius=0.1,
                            grid=synth.azimuth_grid(), drift_deg_per_blk=5.0, seed=4)
    az = np.rad2deg(np.arctan2(w.src_dirs[:, 0, 1], w.src_dirs[:, 0, 0]))
    assert np.allclose(np.mod(np.diff(az), 360.0), 5.0)
    assert np.array_equal(np.diff(w.src_grid_idx[:, 0]) % 72, [1, 1])


def test_fibonacci_direction_set():
    """Golden-angle spiral: unit vectors, equal-area latitude bands (z evenly
    spaced), symmetric neighbour lists without self entries, every direction
    with at least its 6 nearest, all within a few point spacings."""
    ds = synth.fibonacci_sphere(2522)
    assert ds.D == 2522 and ds.n_az == 2522 and ds.n_el == 0
    assert np.allclose(np.linalg.norm(ds.u, axis=1), 1.0)
    assert np.allclose(np.diff(ds.u[:, 2]), -2.0 / 2522)
    ptr, idx = ds.nbr_ptr, ds.nbr_idx
    assert ptr.dtype == np.int32 and idx.dtype == np.int32 and ptr[0] == 0 and ptr[-1] == idx.size
    sets = [set(idx[ptr[d]:ptr[d + 1]].tolist()) for d in range(ds.D)]
    assert all(d not in sets[d] and len(sets[d]) >= 6 for d in range(ds.D))
    assert all(d in sets[n] for d in range(ds.D) for n in sets[d])
    spacing = np.sqrt(4 * np.pi / ds.D)
    ang = [np.arccos(np.clip(ds.u[d] @ ds.u[n], -1, 1)) for d in range(ds.D) for n in sets[d]]
    assert max(ang) < 3 * spacing


def test_grid_neighbour_lists():
    """The 8-neighbourhood of the sphere grid: wrap in azimuth, 5 neighbours
    on the pole rows, 8 inside."""
    ptr, idx = synth.grid_neighbours(72, 19)
    cnt = np.diff(ptr)
    assert cnt[:72].tolist() == [5] * 72 and cnt[72:-72].min() == 8 and cnt[-72:].max() == 5
    assert set(idx[ptr[0]:ptr[1]].tolist()) == {1, 71, 72, 73, 72 + 71}


def test_paper_shape_recipe():
    w = synth.paper_shape(seed=3, nblk=1)
    assert w.X.shape == (1, 50, 73, 60) and w.H.shape == (73, 2522, 60) and w.Ns == 2
    assert np.allclose(w.freqs, 31.25 * np.arange(16, 89))
