"""Batch creation reuses the prologue tables already built in the process
(per device, keyed by cell length and sPAM constants, and by eps_crit for
the wrinkling table): the reused tables are bitwise the built ones, new cell
lengths are built and match the oracle, and other constants get their own
tables."""
import numpy as np
import pytest

import oracle
from paper_2509_15180_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402


def test_reused_tables_are_bitwise_and_new_ones_are_built():
    sc = scenes.parity_batch(16)
    b1 = vine.Batch(sc)
    t1 = b1.tables()
    b2 = vine.Batch(sc)
    t2 = b2.tables()
    for k in ("hdr", "knots", "utab", "consts"):
        assert np.array_equal(t1[k], t2[k]), k
    b1.simulate()
    b2.simulate()
    s1, s2 = b1.state(), b2.state()
    for k in ("theta", "l", "N", "status", "iters"):
        assert np.array_equal(s1[k], s2[k]), k
    # one cell length not seen before (a table to build) beside the cached one
    sc3 = {k: v.copy() for k, v in sc.items()}
    l0_new = np.float32(0.0217)
    sc3["act_l0"][: max(1, sc3["act_l0"].size // 2)] = l0_new
    b3 = vine.Batch(sc3)
    t3 = b3.tables()
    assert t3["n_tab"] == 2
    orc = oracle.Oracle(sc3)
    by_l0 = {np.float32(x[0]): x for x in orc.tables()}
    order = list(dict.fromkeys(np.float32(v) for v in sc3["act_l0"]))  # first appearance, as the batch numbers them
    for t, l0 in enumerate(order):
        _, lo, hi, f = by_l0[l0]
        assert t3["hdr"][t, 0] == pytest.approx(lo, rel=1e-6, abs=1e-9)
        assert np.allclose(t3["knots"][t, :, 0], f, rtol=2e-6, atol=1e-12 * f.max())
    # a different eps_crit gets its own wrinkling table
    p = vine.vine_params_default()
    p.eps_crit = 0.02
    b4 = vine.Batch(sc, p)
    t4 = b4.tables()
    assert not np.array_equal(t4["utab"], t1["utab"])
    assert np.array_equal(t4["hdr"], t1["hdr"]) and np.array_equal(t4["knots"], t1["knots"])
    for b in (b1, b2, b3, b4):
        b.close()
