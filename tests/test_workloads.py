"""The seeded input generators shared by the oracle and the GPU tests (no
method arithmetic): the SplitMix64 stream against the reference generator's
published outputs, and the phantoms, beams and batch jobs against the recipe
they state."""
import numpy as np
import pytest

from paper_0910_0329_gb300 import workloads as W


def test_splitmix64_matches_the_reference_outputs():
    # the reference splitmix64 (Steele, Lea and Flood 2014; Vigna's C version)
    g = W.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    g = W.SplitMix64(1234567)
    assert [g.next_u64() for _ in range(3)] == [6457827717110365317, 3203168211198807973, 9817491932198370423]
    g = W.SplitMix64(6)
    u = [g.uniform() for _ in range(10000)]
    assert all(0.0 <= x < 1.0 for x in u) and abs(np.mean(u) - 0.5) < 0.01


def voxel(ph, i, j, k):
    return i + ph.nx * (j + ph.ny * k)


def test_slab_phantom_layout():
    ph = W.slab_phantom(5, 4, 10, 0.5, [(0, 1.2, W.MAT_WATER, 1.0), (1.2, 3.0, W.MAT_BONE, 1.85),
                                        (3.0, 1e9, W.MAT_LUNG, 0.3)])
    assert ph.n_vox == 200 and ph.extent == (2.5, 2.0, 5.0)
    for k in range(10):
        zc = (k + 0.5) * 0.5
        want = (W.MAT_WATER, 1.0) if zc < 1.2 else (W.MAT_BONE, 1.85) if zc < 3.0 else (W.MAT_LUNG, 0.3)
        for i, j in [(0, 0), (4, 3), (2, 1)]:
            v = voxel(ph, i, j, k)
            assert (ph.mat[v], float(ph.rho[v])) == pytest.approx(want)
    with pytest.raises(ValueError):
        W.slab_phantom(2, 2, 4, 1.0, [(0, 2, W.MAT_WATER, 1.0)])


def test_paper_slab_phantom():
    for middle, m, r in [("bone", W.MAT_BONE, 1.85), ("lung", W.MAT_LUNG, 0.3)]:
        ph = W.paper_slab_phantom(middle)
        assert (ph.nx, ph.ny, ph.nz) == (61, 61, 150) and (ph.dx, ph.dy, ph.dz) == (0.5, 0.5, 0.2)
        col = ph.mat.reshape(150, 61, 61)[:, 30, 30]
        assert list(np.nonzero(col == m)[0]) == list(range(25, 50))  # voxel centres 5.1 .. 9.9 cm
        assert np.all(ph.rho.reshape(150, 61, 61)[25:50] == np.float32(r))
        assert np.all(col[:25] == W.MAT_WATER) and np.all(col[50:] == W.MAT_WATER)


def test_blob_phantom_is_seeded_and_has_three_classes():
    a = W.blob_phantom(64, 64, 64, 0.5, 11)
    b = W.blob_phantom(64, 64, 64, 0.5, 11)
    c = W.blob_phantom(64, 64, 64, 0.5, 12)
    assert np.array_equal(a.mat, b.mat) and np.array_equal(a.rho, b.rho)
    assert not np.array_equal(a.mat, c.mat)
    frac = np.bincount(a.mat, minlength=3) / a.n_vox
    assert frac[W.MAT_WATER] > 0.5 and frac[W.MAT_LUNG] > 0.01 and frac[W.MAT_BONE] > 0.01
    for m, r in [(W.MAT_WATER, 1.0), (W.MAT_LUNG, 0.26), (W.MAT_BONE, 1.85)]:
        assert np.all(a.rho[a.mat == m] == np.float32(r))


def test_axial_source_aims_at_the_phantom_centre():
    wl = W.c1_photon_wbw()
    X, Y, _ = wl.phantom.extent
    s = wl.source
    assert s.iso[0] == pytest.approx(X / 2) and s.iso[1] == pytest.approx(Y / 2)
    # SSD 90 with SAD 100: the isocentre lies 10 cm below the entrance surface
    assert s.iso[2] == pytest.approx(10.0) and s.sad == 100.0


def test_batch_jobs_follow_the_recipe():
    jobs = W.c3_batch(n_jobs=8)
    assert len(jobs) == 8
    sizes = {(64, 64, 64), (96, 96, 96), (128, 128, 128), (256, 256, 128)}
    for i, (ph, src, n, seed) in enumerate(jobs):
        assert (ph.nx, ph.ny, ph.nz) in sizes and 0.2 <= ph.dx <= 0.5
        assert seed == 2000 + i and 10 ** 5 <= n <= 10 ** 7
        if i % 2 == 0:
            assert src.particle == W.PHOTON and src.spectrum == W.SPEC_6MV
        else:
            assert src.particle == W.ELECTRON and src.spectrum == W.SPEC_MONO and 6.0 <= src.energy <= 20.0
    again = W.c3_batch(n_jobs=8)
    assert [(p.name, n, s) for p, _, n, s in jobs] == [(p.name, n, s) for p, _, n, s in again]
