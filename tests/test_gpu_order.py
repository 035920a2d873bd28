"""A robot's result does not depend on where it sits in the batch: the same
robots in another order, and each robot grown alone, give bitwise the same
state for a given team size.  The batch order changes the longest-first
queue, the CTA and shared-memory slice a robot lands on and the slice
layout (sized for the batch's largest robot and obstacle set); none of
these may reach the arithmetic."""
import numpy as np
import pytest

from paper_2509_15180_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402

KEYS = ("N", "l", "tip", "status", "iters", "resid")


def _prm(tp):
    p = vine.vine_params_default()
    p.threads_per_robot = tp
    return p


def _grow(sc, tp):
    b = vine.Batch(sc, _prm(tp))
    b.simulate()
    st = b.state()
    th = [b.theta_of(st, j) for j in range(len(sc["n_links"]))]
    b.close()
    return st, th


def _same(sa, tha, i, sb, thb, j, what):
    for k in KEYS:
        assert np.array_equal(sa[k][i], sb[k][j]), (what, k, i, j)
    assert np.array_equal(tha[i], thb[j]), (what, "theta", i, j)


@pytest.mark.parametrize("tp", [32, 64, 128])
def test_permuted_batch_and_robots_alone_are_bitwise_equal(tp):
    sc = scenes.uneven_batch(48, replicate=5, n_range=(20, 90))
    n = len(sc["n_links"])
    st, th = _grow(sc, tp)
    assert np.count_nonzero(st["N"] == sc["n_links"]) >= n // 2      # the robots did grow
    perm = np.random.default_rng(tp).permutation(n)
    sp, thp = _grow(scenes.subset(sc, perm), tp)
    for j, i in enumerate(perm):
        _same(st, th, i, sp, thp, j, "permuted")
    for i in (int(np.argmax(sc["n_links"])), int(np.argmin(sc["n_links"])), 7):
        sa, tha = _grow(scenes.subset(sc, [i]), tp)
        _same(st, th, i, sa, tha, 0, "alone")
