"""The allocation-free table build (vine_spam_tables_noalloc) against the
tables vine_batch_create builds for the same cell lengths.

Callers that cannot call cudaMalloc (device memory fully handed to another
framework's pool, or latency-critical loops that cannot afford the device
synchronisation of cudaMalloc/cudaFree) use the allocation-free entry point;
its working space is a fixed device array inside the library.  This file is
named to be collected last, so a run that stops at its first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2509_15180_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402

RTOL = 2e-6  # the tolerance of the prologue-table parity test


def _first_appearance(values):
    out = []
    for v in np.asarray(values, dtype=np.float32).astype(np.float64):
        if v not in out:
            out.append(v)
    return np.array(out)


def _reference_tables(sc):
    b = vine.Batch(sc)
    T = b.tables()
    b.close()
    return T


def _noalloc(l0):
    d_l0 = torch.tensor(l0, dtype=torch.float64, device="cuda")
    hdr = torch.zeros((len(l0), 4), dtype=torch.float32, device="cuda")
    knots = torch.zeros((len(l0), 256, 2), dtype=torch.float32, device="cuda")
    vine.vine_spam_tables_noalloc(d_l0, hdr, knots)
    torch.cuda.synchronize()
    return hdr.cpu().numpy(), knots.cpu().numpy()


def test_noalloc_tables_match_batch_tables_on_two_calls():
    # robots with different segment lengths give several distinct cell lengths
    sc1 = scenes.uneven_batch(24, n_range=(30, 40))
    sc2 = scenes.uneven_batch(24, replicate=3, n_range=(30, 40))
    for sc in (sc1, sc2):  # two calls in a row, different inputs
        l0 = _first_appearance(sc["act_l0"])
        assert 2 <= len(l0) <= vine.NOALLOC_MAX_TABLES
        T = _reference_tables(sc)
        assert T["n_tab"] == len(l0)
        hdr, knots = _noalloc(l0)
        assert np.allclose(hdr, T["hdr"], rtol=RTOL, atol=0.0)
        assert np.allclose(knots, T["knots"], rtol=RTOL, atol=1e-12)


def test_noalloc_rejects_more_tables_than_its_scratch_holds():
    l0 = np.full(vine.NOALLOC_MAX_TABLES + 1, 0.02)
    d_l0 = torch.tensor(l0, dtype=torch.float64, device="cuda")
    hdr = torch.zeros((len(l0), 4), dtype=torch.float32, device="cuda")
    knots = torch.zeros((len(l0), 256, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(vine.VineError) as ei:
        vine.vine_spam_tables_noalloc(d_l0, hdr, knots)
    assert ei.value.status == vine.VINE_EINVAL
    assert "n_tab" in vine.last_error()
