"""Parity of the Eq. 26/27 extensions (through the C ABI) with the FP64 oracle:
point detectors (sparse detector rows F of Eq. 27) in every step form, the
sensor response of Eq. 27, the partial-path source column and the sub-step
sources of Section 4.1, and their checkpoint / mode interplay."""

import numpy as np
import pytest

from paper_1611_08536_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_08536_gb300 import build, drts
    build.build()
    drts.load()
    return drts


def rel_l1(a, b):
    return np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300)


def _layered(n=10, precision=I.FP64, n_rhs=1, kernel=0):
    """Two media with different refractive index (interface folding) in a
    Fresnel box, detector patches on +z."""
    mov = np.zeros((n, n, n), np.uint8)
    mov[n // 2:] = 1
    p = I.Problem((n, n, n), 0.1, [(8.0, 0.03, 0.85, 1.4), (4.0, 0.06, 0.7, 1.33)], mov, 1.0,
                  I.FRESNEL, precision, n_rhs, I.FACE_PZ, 2, 2, f"layered{n}")
    p.batched_kernel = kernel
    return p


def _point_rows(prob, seed=0, n_det=6, per=9):
    """n_det detectors of `per` seed-random (state, weight) entries, plus one
    point detector of a single state."""
    rng = np.random.default_rng(seed)
    det = np.repeat(np.arange(n_det - 1), per).astype(np.int32)
    st = rng.integers(0, prob.n_states, det.size).astype(np.int64)
    w = rng.uniform(0.1, 2.0, det.size)
    det = np.r_[det, n_det - 1].astype(np.int32)
    st = np.r_[st, prob.state(prob.shape[0] // 2, prob.shape[1] // 2, prob.shape[2] - 1,
                              I.direction_index(0, 0, 1))]
    w = np.r_[w, 1.0]
    return n_det, det, st, w


def _oracle_point(oracle_mod, prob, csr, steps, src, point):
    return oracle_mod.run(prob, csr, steps, src.as_tuple(), point=point)


@pytest.mark.parametrize("precision,tol", [(I.FP64, 1e-12), (I.FP32, 1e-5)])
def test_point_detectors_match_oracle(gpu, oracle_mod, precision, tol):
    prob = _layered(10, precision)
    src = I.Source(np.array([prob.state(5, 5, 0, I.direction_index(0, 0, 1))], np.int64),
                   np.ones(1), 0, np.ones(1))
    point = _point_rows(prob)
    steps = 60
    csr = oracle_mod.assemble(prob)
    _, deto, _, pdo = _oracle_point(oracle_mod, prob, csr, steps, src, point)
    with gpu.Context(prob, max_steps=steps) as ctx:
        ctx.set_point_detectors(*point)
        ctx.set_source(0, src)
        ctx.step_n(steps)
        pd = ctx.read_point_detectors()
        det, _ = ctx.read_detectors()
    assert pd.shape == pdo.shape
    for d in range(point[0]):
        assert rel_l1(pd[:, d], pdo[:, d]) < tol, d
    assert rel_l1(det, deto) < tol


def test_point_detectors_with_exit_weights_equal_face_detector(gpu, oracle_mod):
    """F = exit coefficient over each face patch reproduces the face detector."""
    prob = _layered(8, I.FP64)
    ab, ex, ed, patch = oracle_mod.column_info(prob)
    sel = np.flatnonzero((patch >= 0) & (ed > 0))
    src = I.Source(np.array([prob.state(4, 4, 0, I.direction_index(0, 0, 1))], np.int64),
                   np.ones(1), 0, np.ones(1))
    with gpu.Context(prob, max_steps=40) as ctx:
        ctx.set_point_detectors(int(patch.max()) + 1, patch[sel], sel, ed[sel])
        ctx.set_source(0, src)
        ctx.step_n(40)
        pd = ctx.read_point_detectors()
        det, _ = ctx.read_detectors()
    assert det.any()
    np.testing.assert_allclose(pd, det, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("kernel,n_rhs", [(0, 5), (1, 8)])
def test_point_detectors_batched(gpu, oracle_mod, kernel, n_rhs):
    """CUDA-core and tensor-core batched steps, one history per right-hand side."""
    prob, srcs = I.inclusions(10, n_rhs=n_rhs, seed=4, precision=I.FP32, n_spheres=1)
    prob.batched_kernel = kernel
    point = _point_rows(prob, seed=3)
    steps = 30
    csr = oracle_mod.assemble(prob)
    with gpu.Context(prob, max_steps=steps) as ctx:
        ctx.set_point_detectors(*point)
        for r, s in enumerate(srcs):
            ctx.set_source(r, s)
        ctx.step_n(steps)
        pds = [ctx.read_point_detectors(r) for r in range(n_rhs)]
    for r in (0, n_rhs // 2, n_rhs - 1):
        _, _, _, pdo = _oracle_point(oracle_mod, prob, csr, steps, srcs[r], point)
        tol = 1e-5 if kernel == 0 else 1e-4
        assert rel_l1(pds[r], pdo) < tol, r


def test_point_detectors_persistent_mode(gpu, oracle_mod):
    prob = _layered(10, I.FP64)
    src = I.Source(np.array([prob.state(5, 5, 0, I.direction_index(0, 0, 1))], np.int64),
                   np.ones(1), 0, np.ones(1))
    point = _point_rows(prob, seed=7)
    steps = 50
    csr = oracle_mod.assemble(prob)
    _, _, _, pdo = _oracle_point(oracle_mod, prob, csr, steps, src, point)
    with gpu.Context(prob, max_steps=steps) as ctx:
        ctx.set_point_detectors(*point)
        ctx.set_source(0, src)
        ctx.set_step_mode(gpu.STEP_PERSISTENT)
        ctx.step_n(20)
        ctx.step_n(steps - 20)
        pd = ctx.read_point_detectors()
    for d in range(point[0]):
        assert rel_l1(pd[:, d], pdo[:, d]) < 1e-12, d


def test_point_detectors_checkpoint_resume(gpu):
    prob = _layered(8, I.FP32)
    src = I.Source(np.array([prob.state(4, 4, 0, I.direction_index(0, 0, 1))], np.int64),
                   np.ones(1), 0, np.ones(1))
    point = _point_rows(prob, seed=9)
    with gpu.Context(prob, max_steps=40) as ctx:
        ctx.set_point_detectors(*point)
        ctx.set_source(0, src)
        ctx.step_n(40)
        ref = ctx.read_point_detectors()
    with gpu.Context(prob, max_steps=40) as ctx:
        ctx.set_point_detectors(*point)
        ctx.set_source(0, src)
        ctx.step_n(15)
        blob = ctx.checkpoint()
    with gpu.Context(prob, max_steps=40) as ctx:
        ctx.set_source(0, src)
        with pytest.raises(gpu.DrtsError):
            ctx.restore(blob)                 # point detectors not set yet
        ctx.set_point_detectors(*point)
        ctx.restore(blob)
        ctx.step_n(25)
        got = ctx.read_point_detectors()
    assert np.array_equal(got, ref)


def test_point_detectors_invalid(gpu):
    prob = _layered(6, I.FP64)
    with gpu.Context(prob, max_steps=5) as ctx:
        for bad in [(2, [2], [0], [1.0]), (2, [0], [prob.n_states], [1.0]), (2, [0], [0], [np.nan])]:
            with pytest.raises(gpu.DrtsError):
                ctx.set_point_detectors(*bad)
        ctx.set_point_detectors(1, [0], [0], [1.0])
        with pytest.raises(gpu.DrtsError):
            ctx.step_n(6)                     # history holds max_steps steps
    with gpu.Context(prob, max_steps=0) as ctx:
        with pytest.raises(gpu.DrtsError):
            ctx.set_point_detectors(1, [0], [0], [1.0])


# --------------------------------------------------------------------------
# Eq. 27 sensor response


@pytest.mark.parametrize("which", [0, 1])
def test_sensor_response_matches_oracle(gpu, oracle_mod, which):
    """The sensor kernel applied to the recorded history equals the oracle's
    sensor response of the same history, bit for bit (same order, no
    contraction)."""
    prob = _layered(8, I.FP64)
    src = I.Source(np.array([prob.state(4, 4, 0, I.direction_index(0, 0, 1))], np.int64),
                   np.ones(1), 0, np.ones(1))
    point = _point_rows(prob, seed=11)
    w = 4
    lags = np.arange(-w, w + 1)
    h = np.where(lags >= 0, np.exp(-lags / 1.5), 0.0)
    with gpu.Context(prob, max_steps=50) as ctx:
        ctx.set_point_detectors(*point)
        ctx.set_source(0, src)
        ctx.step_n(50)
        D = ctx.read_detectors()[0] if which == 0 else ctx.read_point_detectors()
        M = ctx.sensor_response(w, h, which=which)
        Mpart = ctx.sensor_response(w, h, which=which, t_begin=10, t_end=30)
    Mo = oracle_mod.sensor_response(D, w, h)
    assert np.array_equal(M, Mo)
    assert np.array_equal(Mpart, Mo[10:30])


# --------------------------------------------------------------------------
# Section 4.1: partial-path source column and sub-step sources


def test_source_column_matches_oracle(gpu, oracle_mod):
    prob = _layered(8, I.FP64)
    D = I.direction_index
    cases = [(4, 4, 0, D(0, 0, 1)), (0, 0, 0, D(-1, -1, -1)), (3, 5, 3, D(0, 1, 1)),
             (3, 3, 4, D(0, 0, 1)), (7, 2, 7, D(1, 0, 0))]
    with gpu.Context(prob, max_steps=0) as ctx:
        assert ctx.substep_count(prob.state(1, 1, 1, 0)) == 2
        for (x, y, z, d) in cases:
            s = prob.state(x, y, z, d)
            for frac in (0.25, 0.5, 0.75, 1.0):
                st, val, ex = ctx.source_column(s, frac)
                sto, valo, exo = oracle_mod.source_column(prob, s, frac)
                assert st.tolist() == sto.tolist(), (x, y, z, d, frac)
                np.testing.assert_allclose(val, valo, rtol=1e-13)
                assert ex == pytest.approx(exo, rel=1e-12, abs=1e-300)


def _substep_oracle(oracle_mod, prob, csr, steps, state, weight, t0, prof):
    """Superposition over sub-intervals: each is a plain source whose entries
    are the oracle's partial-path column."""
    n_sub = prof.shape[1]
    x = np.zeros(prob.n_states)
    det = None
    led = np.zeros(4)
    for j in range(n_sub):
        st, val, _ = oracle_mod.source_column(prob, state, 1.0 - (j + 0.5) / n_sub)
        xj, dj, lj = oracle_mod.run(prob, csr, steps, (st, weight * val, t0, prof[:, j]))
        x += xj
        det = dj if det is None else det + dj
        led += lj
    return x, det, led


@pytest.mark.parametrize("precision,tol", [(I.FP64, 1e-12), (I.FP32, 1e-5)])
def test_substep_source_matches_oracle(gpu, oracle_mod, precision, tol):
    prob = _layered(10, precision)
    state = prob.state(5, 5, 0, I.direction_index(0, 0, 1))
    t0, g = I.gaussian_profile(3.0)
    # split each step's emission over its two dr/c sub-intervals, 40 / 60
    prof = np.stack([0.4 * g, 0.6 * g], 1)
    steps = 40
    csr = oracle_mod.assemble(prob)
    xo, deto, ledo = _substep_oracle(oracle_mod, prob, csr, steps, state, 1.5, t0, prof)
    with gpu.Context(prob, max_steps=steps) as ctx:
        assert ctx.substep_count(state) == 2
        ctx.inject_source_substeps(0, [state], [1.5], t0, prof)
        ctx.step_n(steps)
        x = ctx.read_state()
        det, led = ctx.read_detectors()
    assert rel_l1(x, xo) < tol
    assert rel_l1(det, deto) < tol
    np.testing.assert_allclose(led, ledo, rtol=max(tol, 1e-11))


def test_substep_and_plain_sources_add_batched(gpu, oracle_mod):
    """Batched FP32 step: rhs 0 plain source only, rhs 1 sub-step only, rhs 2
    both (linearity)."""
    prob, srcs = I.inclusions(10, n_rhs=3, seed=12, precision=I.FP32, n_spheres=1)
    state = prob.state(5, 4, 0, I.direction_index(0, 1, 1))
    prof = np.array([[0.5, 0.5], [0.2, 0.1]])
    steps = 30
    csr = oracle_mod.assemble(prob)
    with gpu.Context(prob, max_steps=steps) as ctx:
        ctx.set_source(0, srcs[0])
        ctx.inject_source_substeps(1, [state], [1.0], 2, prof)
        ctx.set_source(2, srcs[2])
        ctx.inject_source_substeps(2, [state], [1.0], 2, prof)
        ctx.step_n(steps)
        xs = [ctx.read_state(r) for r in range(3)]
    xsub, _, _ = _substep_oracle(oracle_mod, prob, csr, steps, state, 1.0, 2, prof)
    x0, _, _ = oracle_mod.run(prob, csr, steps, srcs[0].as_tuple())
    x2, _, _ = oracle_mod.run(prob, csr, steps, srcs[2].as_tuple())
    assert rel_l1(xs[0], x0) < 1e-5
    assert rel_l1(xs[1], xsub) < 1e-5
    assert rel_l1(xs[2], x2 + xsub) < 1e-5


def test_substep_source_mode_limits(gpu):
    prob = _layered(6, I.FP64)
    state = prob.state(3, 3, 0, I.direction_index(0, 0, 1))
    with gpu.Context(prob, max_steps=10) as ctx:
        ctx.inject_source_substeps(0, [state], [1.0], 0, np.ones((1, 2)))
        with pytest.raises(gpu.DrtsError):
            ctx.set_step_mode(gpu.STEP_PERSISTENT)
        with pytest.raises(gpu.DrtsError):
            ctx.run_host(np.ones((2, 1)))
        with pytest.raises(gpu.DrtsError):
            ctx.inject_source_substeps(0, [state], [1.0], 0, np.ones((1, 65)))
        ctx.inject_source_substeps(0, [], [], 0, np.ones((1, 2)))      # removes it
        ctx.set_step_mode(gpu.STEP_PERSISTENT)
        ctx.step_n(2)


def test_point_detectors_replaced_and_kept_on_error(gpu, oracle_mod):
    """Setting detectors again replaces the set and clears its history (steps
    before the call read 0); a rejected call leaves the current set alone."""
    prob = _layered(8, I.FP64)
    src = I.Source(np.array([prob.state(4, 4, 0, I.direction_index(0, 0, 1))], np.int64),
                   np.ones(1), 0, np.ones(1))
    first, second = _point_rows(prob, seed=1, n_det=3), _point_rows(prob, seed=2, n_det=5)
    csr = oracle_mod.assemble(prob)
    _, _, _, pdo = _oracle_point(oracle_mod, prob, csr, 12, src, second)
    with gpu.Context(prob, max_steps=12) as ctx:
        ctx.set_source(0, src)
        ctx.set_point_detectors(*first)
        ctx.step_n(5)
        ctx.set_point_detectors(*second)
        with pytest.raises(gpu.DrtsError):
            ctx.set_point_detectors(2, [5], [0], [1.0])        # detector index out of range
        ctx.step_n(7)
        pd = ctx.read_point_detectors()
    assert pd.shape == (12, 5)
    assert not pd[:5].any()
    np.testing.assert_allclose(pd[5:], pdo[5:], rtol=1e-12, atol=1e-300)


def test_substep_source_replaced(gpu, oracle_mod):
    """A second sub-step source for the same rhs replaces the first."""
    prob = _layered(8, I.FP64)
    s1 = prob.state(4, 4, 0, I.direction_index(0, 0, 1))
    s2 = prob.state(3, 5, 0, I.direction_index(1, 0, 1))
    prof = np.array([[0.3, 0.7]])
    csr = oracle_mod.assemble(prob)
    xo, _, _ = _substep_oracle(oracle_mod, prob, csr, 10, s2, 2.0, 0, prof)
    with gpu.Context(prob, max_steps=10) as ctx:
        ctx.inject_source_substeps(0, [s1], [1.0], 0, prof)
        ctx.inject_source_substeps(0, [s2], [2.0], 0, prof)
        ctx.step_n(10)
        x = ctx.read_state()
    assert rel_l1(x, xo) < 1e-12
