"""The seeded input recipes: the generator against its published definition,
and each workload against the distributions and sizes its docstring states."""
import math

import numpy as np

from paper_2403_11636_gb300 import inputs


def test_splitmix64_reference_outputs():
    """First outputs of SplitMix64 (Steele, Lea, Flood 2014) as printed by the
    reference implementation for seeds 0 and 1234567."""
    r = inputs.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    r = inputs.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(3)] == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_uniform_array_is_the_scalar_stream():
    seed = 0xABCDEF
    r = inputs.SplitMix64(seed)
    want = np.array([r.uniform(-1.0, 1.0) for _ in range(1000)])
    np.testing.assert_array_equal(inputs.uniform_array(1000, seed), want)
    u = inputs.uniform_array(100000, 3)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01


def test_porous_3d_recipe():
    """40 non-overlapping spheres inside the unit cube, radii in [0.04, 0.12],
    64^3 cells, 5 levels, alpha 1e-8, octree depth 3, walls on y/z faces."""
    for seed in (0, 1, 7):
        p = inputs.porous_3d(seed)
        s = p.shapes
        assert s.shape == (40, 9) and np.all(s[:, 0] == 0.0)
        r, c = s[:, 4], s[:, 1:4]
        assert r.min() >= 0.04 and r.max() <= 0.12
        assert np.all(c - r[:, None] >= 0.0) and np.all(c + r[:, None] <= 1.0)
        d = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=2)
        rr = r[:, None] + r[None, :]
        assert np.all(d[~np.eye(40, dtype=bool)] >= rr[~np.eye(40, dtype=bool)])
        assert (p.n, p.nlevels, p.alpha, p.qdepth, p.preset) == ((64, 64, 64), 5, 1e-8, 3, 1)
        assert p.ndof() == 65 ** 3 * 4 == 1098500
    assert not np.array_equal(inputs.porous_3d(0).shapes, inputs.porous_3d(1).shapes)
    np.testing.assert_array_equal(inputs.porous_3d(5).shapes, inputs.porous_3d(5).shapes)


def test_radius_scale_keeps_the_solid_fraction():
    """The scale holds the expected solid fraction at 30 % once U[0.04, 0.12]
    radii would exceed it (0.720 for 300 spheres); below that it is 1."""
    assert inputs.radius_scale(40) == 1.0
    s = inputs.radius_scale(300)
    assert abs(s - 0.720) < 5e-4
    rmin, rmax = 0.04 * s, 0.12 * s
    e_r3 = (rmax ** 4 - rmin ** 4) / (4 * (rmax - rmin))
    assert abs(300 * 4.0 / 3.0 * math.pi * e_r3 - 0.30) < 1e-12


def test_batch_2d_recipe():
    """Grids from {16, 32, 64, 128}^2, 1-8 ellipses with semi-axes in
    [0.03, 0.2], centres in [0.25, 0.75]^2, alpha from {1e-6, 1e-8, 1e-10},
    levels halved down to 4^2 cells; the 256-problem batch holds 4,138,464
    DoFs and 1,379,488 finest-level patches."""
    ps = [inputs.batch_2d(s) for s in range(256)]
    assert {p.n[0] for p in ps} == {16, 32, 64, 128}
    assert {len(p.shapes) for p in ps} == set(range(1, 9))
    assert {p.alpha for p in ps} == {1e-6, 1e-8, 1e-10}
    for p in ps:
        assert p.n[0] == p.n[1] and p.n[0] >> (p.nlevels - 1) == 4
        s = p.shapes
        assert np.all(s[:, 0] == 1.0)
        assert np.all((s[:, 1:3] >= 0.25) & (s[:, 1:3] <= 0.75))
        assert np.all((s[:, 4:6] >= 0.03) & (s[:, 4:6] <= 0.2))
        np.testing.assert_allclose(s[:, 7] ** 2 + s[:, 8] ** 2, 1.0, rtol=0, atol=1e-15)
        assert np.all(s[:, 8] >= 0.0)           # angle in [0, pi)
    assert sum(p.ndof() for p in ps) == 4138464
    assert sum((p.n[0] + 1) * (p.n[1] + 1) for p in ps if p.nlevels > 1) == 1379488


def test_channel_workloads():
    p = inputs.channel_2d(3)
    cx, cy = p.shapes[0, 1:3]
    assert 0.35 <= cx <= 0.65 and 0.35 <= cy <= 0.65 and p.shapes[0, 4] == 0.2
    q = inputs.channel_replay_2d(0)
    assert (q.n, q.hi, q.nu_pre, q.nu_post) == ((1024, 256), (2.2, 0.41), 6, 6)
    assert q.shapes[0, 4] == 0.05                # cylinder diameter 0.1
    assert 0.15 <= q.shapes[0, 1] <= 0.25 and 0.15 <= q.shapes[0, 2] <= 0.26
    assert q.ndof() == 790275                    # the paper's coarse grid (Table tab:grid)
