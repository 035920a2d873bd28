"""Launch autotuner (vine_autotune): it times every candidate launch
configuration on a sample, adopts the fastest, and changes no result."""
import numpy as np
import pytest

from paper_2509_15180_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402


def test_autotune_picks_a_candidate_and_keeps_results():
    sc = scenes.uneven_batch(192, n_range=(30, 120))
    b = vine.Batch(sc)
    b.simulate()
    ref = b.state()
    r = b.autotune(sample=96)
    print("autotune:", r)
    assert r["candidates"] >= 3 and r["sample"] == 96
    assert r["warps_per_cta"] in (1, 2, 4) and r["list_margin"] in (0.5, 1.0, 2.0)
    assert 0.0 < r["best_ms"] <= r["default_ms"] or r["default_ms"] < 0
    st = b.state()
    assert np.all(st["N"] == 0)  # left reset
    b.simulate()
    st = b.state()
    for k in ("theta", "l", "N", "status", "iters", "resid"):
        assert np.array_equal(st[k], ref[k]), k
    b.close()
