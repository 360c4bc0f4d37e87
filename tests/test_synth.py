"""The seeded scene generator: shapes, determinism, and the camera model."""
import numpy as np

import synth


def test_shapes_and_determinism():
    spec = synth.SceneSpec(40, 24, (0.25, 1.0, 4.0), d_max=4)
    a = synth.make_stack(spec, 5)
    b = synth.make_stack(spec, 5)
    c = synth.make_stack(spec, 6)
    assert a.shape == (6, 24, 40, 3) and a.dtype == np.uint8
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_irradiance_dynamic_range_and_exposure_order():
    spec = synth.SceneSpec(64, 48, (0.25, 1.0, 4.0))
    rng = np.random.Generator(np.random.PCG64(1))
    E = synth._irradiance(rng, spec)
    assert abs(E.max() / E.min() - 2.0 ** 12) < 1e-6 * 2.0 ** 12
    assert abs(np.exp(np.mean(np.log(E))) - 0.18) < 1e-12
    img = synth.make_stack(spec, 1).astype(int)
    # longer exposure never darkens a pixel (same view)
    assert np.all(img[1] >= img[0]) and np.all(img[2] >= img[1])
    assert np.all(img[4] >= img[3]) and np.all(img[5] >= img[4])


def test_right_view_is_shifted_left_view():
    spec = synth.SceneSpec(64, 48, (1.0,), d_max=0)
    img = synth.make_stack(spec, 2)
    assert np.array_equal(img[0], img[1])   # zero disparity: identical views


def test_named_workloads():
    for name in synth.CONFIGS:
        cfg = synth.config_spec(name)
        spec = cfg["spec"]
        assert len(cfg["ranks"]) == 4
        assert cfg["ranks"][2] <= 3 and cfg["ranks"][3] <= spec.K
    assert synth.seed_for("small_64x48", 3) == 1003
