"""Length classes and the launch autotuner (vine_autotune).

A batch grows in length classes (robots of up to 64 links, 65-200, more),
each a persistent launch of its own team size on a parallel branch of the
CUDA graph.  A robot's result then depends only on its own length, not on
the batch it is in.  The autotuner times team sizes per class and the
broad-phase margin on a sample, adopts the tuned configuration only if the
sample grows faster, and every robot's result is then bitwise the one of a
batch grown with its class's chosen team size (the margin changes nothing)."""
import numpy as np
import pytest

from paper_2509_15180_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402

KEYS = ("l", "N", "status", "iters", "resid")


def _same_robot(s1, b1, i1, s2, b2, i2):
    assert np.array_equal(b1.theta_of(s1, i1), b2.theta_of(s2, i2)), (i1, i2)
    for k in KEYS:
        assert s1[k][i1] == s2[k][i2] or (np.isnan(s1[k][i1]) and np.isnan(s2[k][i2])), (k, i1, i2)


def _grown_with(sc, idx, tp):
    p = vine.vine_params_default()
    p.threads_per_robot = tp
    b = vine.Batch(scenes.subset(sc, idx), p)
    b.simulate()
    return b, b.state()


def test_length_classes_and_robot_results_independent_of_the_batch():
    sc = scenes.uneven_batch(96, replicate=3, n_range=(30, 300))
    b = vine.Batch(sc)
    cls = b.classes()
    assert [c["threads_per_robot"] for c in cls] == [128, 64, 32]
    nl = sc["n_links"]
    assert [c["robots"] for c in cls] == [int((nl > 200).sum()), int(((nl > 64) & (nl <= 200)).sum()),
                                          int((nl <= 64).sum())]
    assert [c["max_links"] for c in cls] == [int(nl[nl > 200].max()), int(nl[(nl > 64) & (nl <= 200)].max()),
                                             int(nl[nl <= 64].max())]
    b.simulate()
    st = b.state()
    # robots grown in batches of their own class, and alone, give bitwise the same
    for tp, sel in ((128, nl > 200), (64, (nl > 64) & (nl <= 200)), (32, nl <= 64)):
        idx = np.nonzero(sel)[0]
        bc, sc_ = _grown_with(sc, idx, tp)
        for k, i in enumerate(idx):
            _same_robot(st, b, i, sc_, bc, k)
        bc.close()
        i = int(idx[0])
        ba = vine.Batch(scenes.subset(sc, [i]))
        ba.simulate()
        _same_robot(st, b, i, ba.state(), ba, 0)
        ba.close()
    b.close()


def test_autotune_tunes_threads_per_robot_per_class():
    sc = scenes.uneven_batch(192, replicate=4, n_range=(30, 300))
    b = vine.Batch(sc)
    r = b.autotune(sample=96)
    print("autotune:", r)
    assert r["n_class"] == 3 and r["sample"] >= 96
    assert r["candidates"] >= 1 + 3 * 3 + 3  # default, per class >= 3 team shapes, 3 margins
    assert r["list_margin"] in (0.5, 1.0, 2.0)
    assert r["default_ms"] > 0.0 and 0.0 < r["best_ms"] <= r["default_ms"]
    assert all(t in (32, 64, 128) for t in r["class_threads"])
    assert [c["threads_per_robot"] for c in b.classes()] == r["class_threads"]
    st = b.state()
    assert np.all(st["N"] == 0)  # left reset
    b.simulate()
    st = b.state()
    nl = sc["n_links"]
    for c, sel in enumerate((nl > 200, (nl > 64) & (nl <= 200), nl <= 64)):
        idx = np.nonzero(sel)[0]
        bc, sc_ = _grown_with(sc, idx, r["class_threads"][c])
        for k, i in enumerate(idx):
            _same_robot(st, b, i, sc_, bc, k)
        bc.close()
    b.close()
