"""The funnelling and robustness statistics on point sets whose answer is
known."""
import numpy as np
import pytest

from paper_2509_15180_gb300 import analysis


def test_density_of_a_square_grid_is_exact():
    # unit grid, k = 4: every interior point has its 4 nearest neighbours at
    # distance 1, so p = 4 / pi there
    g = np.stack(np.meshgrid(np.arange(12.0), np.arange(12.0)), -1).reshape(-1, 2)
    p = analysis.knn_densities(g, 4)
    inner = (g[:, 0] > 0) & (g[:, 0] < 11) & (g[:, 1] > 0) & (g[:, 1] < 11)
    assert np.allclose(p[inner], 4.0 / np.pi)


def test_concentration_ratio_grows_with_clustering():
    rng = np.random.default_rng(1)
    even = np.stack(np.meshgrid(np.linspace(0, 1, 10), np.linspace(0, 1, 10)), -1).reshape(-1, 2)
    r_even = analysis.density_concentration_ratio(even + 1e-9 * rng.standard_normal(even.shape), k=4)
    clustered = np.concatenate([rng.normal(0.5, 0.5, (80, 2)), rng.normal(0.2, 0.005, (20, 2))])
    r_cl = analysis.density_concentration_ratio(clustered, k=4)
    assert 1.0 <= r_even < 1.3
    assert r_cl > 5.0 * r_even


def test_success_rate():
    tips = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0]])
    goals = np.zeros((3, 2))
    assert analysis.success_rate(tips, goals, 1.0) == pytest.approx(2.0 / 3.0)
    with pytest.raises(ValueError):
        analysis.knn_densities(tips, 3)


def test_study_scenes_are_seeded_and_shaped():
    from paper_2509_15180_gb300 import scenes
    nom = scenes.nominal_design()
    a, la = scenes.robustness_sweep(nom, (0.0, 0.05, 0.1), trials=7, kind="obstacles")
    b, lb = scenes.robustness_sweep(nom, (0.0, 0.05, 0.1), trials=7, kind="obstacles")
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(la, np.repeat([0, 1, 2], 7))
    # level 0 leaves the design untouched; higher levels move the obstacles
    o = slice(int(a["obs_ptr"][0]), int(a["obs_ptr"][1]))
    assert np.array_equal(a["obs_cx"][o], nom["obs_cx"])
    o7 = slice(int(a["obs_ptr"][14]), int(a["obs_ptr"][15]))
    assert not np.array_equal(a["obs_cx"][o7], nom["obs_cx"])
    c, _ = scenes.robustness_sweep(nom, (0.0, 0.2), trials=3, kind="actuation")
    assert np.array_equal(c["act_pressure"][:2], nom["act_pressure"])
    assert np.all(c["act_end"] > c["act_begin"]) and np.all(c["act_pressure"] >= 0)
    f, env = scenes.funnel_rollouts(n_rollouts=10, counts=(0, 5))
    assert np.array_equal(np.bincount(env), [10, 10])
    heads = f["base"][:, 2]
    assert np.all(np.abs(heads) <= 0.3) and np.unique(heads).size == 20
