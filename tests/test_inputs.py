"""The seeded synthetic workloads (paper_1611_08536_gb300/inputs.py) follow
their stated recipes: sizes, media, sources, pulse profiles, arrival process,
and they are reproducible from their seeds.  CPU only."""
import math
import os

import numpy as np
import pytest

from paper_1611_08536_gb300 import inputs as I


def _voxel_dir(prob, s):
    v, d = divmod(int(s), 26)
    nx, ny, _ = prob.shape
    return (v % nx, v // nx % ny, v // (nx * ny)), I.direction_vector(d)


def test_fresnel_cube_recipe():
    prob, src = I.fresnel_cube(16)
    assert prob.shape == (16, 16, 16) and prob.voxel_mm == 0.1
    assert prob.media == [(10.0, 0.01, 0.9, 1.4)] and prob.boundary == I.FRESNEL
    assert prob.n_outside == 1.0 and prob.precision == I.FP64
    (c, v), = [_voxel_dir(prob, s) for s in src.state]
    assert c == (8, 8, 0) and tuple(v) == (0, 0, 1)
    assert list(src.profile) == [1.0] and src.t0 == 0


def test_three_layers_recipe():
    prob, src = I.three_layers(128)
    mov = np.asarray(prob.medium_of_voxel)
    thickness = [int((mov[:, 0, 0] == k).sum()) for k in range(3)]
    assert thickness == [11, 21, 96]                        # 1 : 2 : 9 mm of 12 mm
    assert np.all(mov == mov[:, :1, :1])                     # planar layers along z
    assert prob.voxel_mm == pytest.approx(12.0 / 128)
    assert [m[3] for m in prob.media] == [1.45, 1.44, 1.37]
    assert (prob.det_face, prob.det_nu, prob.det_nv) == (I.FACE_PZ, 16, 16)
    (c, v), = [_voxel_dir(prob, s) for s in src.state]
    assert c == (64, 64, 0) and tuple(v) == (0, 0, 1)
    # Gaussian FWHM 3 steps, centre 2 FWHM, support +-3 FWHM, sum 1 (reading R10)
    t = src.t0 + np.arange(len(src.profile))
    assert src.profile.sum() == pytest.approx(1.0, rel=1e-15)
    assert t[np.argmax(src.profile)] == 6 and t[0] == 0 and t[-1] == 15
    p = dict(zip(t.tolist(), src.profile))
    half = p[6] / 2
    assert p[5] > half > p[4] and p[7] > half > p[8]         # full width at half maximum: 3 steps
    assert p[5] == pytest.approx(p[7], rel=1e-15)


def test_inclusions_recipe():
    prob, srcs = I.inclusions(96, 64)
    mov = np.asarray(prob.medium_of_voxel)
    assert prob.media[1][1] == pytest.approx(10 * prob.media[0][1])      # mu_a x 10
    assert prob.media[1][0] == prob.media[0][0] and prob.media[1][3] == prob.media[0][3]
    frac = mov.mean()
    vol = [4 / 3 * math.pi * r ** 3 for r in (4, 10)]
    assert 0 < frac * 96 ** 3 <= 4 * vol[1] * 1.1              # four spheres of radius <= 10
    assert len(srcs) == 64
    for s in srcs:
        (c, v), = [_voxel_dir(prob, st) for st in s.state]
        on = [a for a in range(3) if c[a] in (0, 95)]
        assert on, c                                            # a surface voxel
        # the direction points into the medium on (at least) one face it sits on
        assert any((v[a] > 0 if c[a] == 0 else v[a] < 0) for a in on)


def test_ellipsoids_recipe():
    prob, src = I.ellipsoids(64, n_ell=12)
    assert len(prob.media) == 13
    for mu_s, mu_a, g, n in prob.media[1:]:
        assert 5.0 <= mu_s <= 30.0 and 0.002 <= mu_a <= 0.05 and 0.7 <= g <= 0.95
        assert 1.33 <= n <= 1.5 and round(n, 3) == n
    assert prob.det_nu == prob.det_nv == 64                     # full exit-face readout


def test_served_stream_recipe():
    reqs = I.served_stream(40, 50.0)
    arr = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(arr) > 0)
    assert 0.5 / 50 < np.mean(np.diff(arr)) < 2.0 / 50           # Poisson at 50/s
    for r in reqs:
        n = r.problem.shape[0]
        assert r.problem.shape == (n, n, n) and n in I.SERVED_SIDES
        assert 500 <= r.n_steps <= 3000
        assert 1 <= len(r.sources) == r.problem.n_rhs <= 16
        for mu_s, mu_a, g, nr in r.problem.media:
            assert 1.0 <= mu_s <= 30.0 and 0.001 <= mu_a <= 0.1 and 0.7 <= g <= 0.95
            assert 1.33 <= nr <= 1.5


def test_workloads_are_reproducible_from_their_seeds():
    a, sa = I.inclusions(24, 8, seed=9)
    b, sb = I.inclusions(24, 8, seed=9)
    c, _ = I.inclusions(24, 8, seed=10)
    assert np.array_equal(a.medium_of_voxel, b.medium_of_voxel)
    assert [list(s.state) for s in sa] == [list(s.state) for s in sb]
    assert not np.array_equal(a.medium_of_voxel, c.medium_of_voxel)
    r1 = I.served_request(4, 7)
    r2 = I.served_request(4, 7)
    assert r1.problem.media == r2.problem.media and r1.n_steps == r2.n_steps
    assert np.array_equal(r1.problem.medium_of_voxel, r2.problem.medium_of_voxel)


def test_config_files_build_their_workloads():
    """Each JSON problem file names a generator, its seeds, a precision and a
    step count; loading it gives the same problem as calling the generator
    (sizes, media map, sources), at the configurations' sizes."""
    names = I.config_names()
    assert names == ["batched_inclusions96x64", "large_ellipsoids192", "plain_fp32_three_layers128",
                     "plain_fp64_cube16", "served_stream1000"]
    c = I.load_config("plain_fp64_cube16")
    p, s = I.fresnel_cube(16, precision=I.FP64)
    assert c.problem.n_states == 106496 and c.steps == 300 and c.problem.precision == I.FP64
    assert np.array_equal(c.sources[0].state, s.state)
    c = I.load_config("batched_inclusions96x64", precision="fp16")
    p, srcs = I.inclusions(96, n_rhs=64, seed=3, precision=I.FP16_ROWSCALE)
    assert c.problem.shape == (96, 96, 96) and c.problem.n_rhs == 64 and len(c.sources) == 64
    assert c.problem.precision == I.FP16_ROWSCALE and c.steps == 1500
    assert np.array_equal(c.problem.medium_of_voxel, p.medium_of_voxel)
    assert all(np.array_equal(a.state, b.state) for a, b in zip(c.sources, srcs))
    c = I.load_config("plain_fp32_three_layers128")
    assert c.problem.n_states == 26 * 128 ** 3 and c.steps == 2000
    assert (c.problem.det_nu, c.problem.det_nv) == (16, 16)
    c = I.load_config("served_stream1000")
    assert c.problem is None and len(c.requests) == 1000
    assert {r.problem.shape[0] for r in c.requests} == {32, 48, 64, 80, 96}
    assert all(500 <= r.n_steps <= 3000 and 1 <= len(r.sources) <= 16 for r in c.requests)
    spec = I.load_config(os.path.join(I.CONFIG_DIR, "large_ellipsoids192.json")).spec
    assert spec["steps"] == 5000 and spec["step_mode"] == "persistent" and spec["args"]["n_ell"] == 12
    with pytest.raises(ValueError):
        I.load_config("plain_fp64_cube16", precision="fp8")
