"""The analysis workloads of Sec. 6.3 / 6.4 (robustness sweep, funnelling
rollouts) on the GPU against the oracle: every robot of a small version of
each study, grown in one launch, against the oracle's growth of the same
robot (poses and contact sets within the parity bar, or a validated switch
at a snap-through); the statistics then follow from the same tips."""
import numpy as np
import pytest

import oracle
from paper_2509_15180_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import studies, vine  # noqa: E402
from test_gpu_parity import _check_switches, _classify  # noqa: E402


def _against_oracle(sc):
    b = vine.Batch(sc)
    b.simulate()
    st = b.state()
    counts, pairs = b.contacts(1024)
    orc = oracle.Oracle(sc, oracle.default_params(tol=1e-10))
    ost = orc.new_state()
    orc.run(ost, int(sc["n_links"].max()), threads=16)
    cls = _classify(b, st, orc, ost, sc, counts, pairs)
    first = _check_switches(b, st, sc, cls)
    b.close()
    return cls, first


@pytest.mark.parametrize("kind", ["obstacles", "actuation"])
def test_robustness_sweep_small_against_oracle(kind):
    nom = scenes.nominal_design()
    sc, lev = scenes.robustness_sweep(nom, (0.0, 0.1, 0.2), trials=24, kind=kind)
    cls, first = _against_oracle(sc)
    print("robustness %s: %d match, %d switches (parting at %s), %d flagged" % (
        kind, cls.count("match"), cls.count("switch"), first, cls.count("flagged")))
    assert cls.count("flagged") <= 2
    # level 0 is the nominal design itself, 24 times: identical robots
    assert all(c == "match" for c, l in zip(cls, lev) if l == 0)


def test_funnel_rollouts_small_against_oracle():
    sc, env = scenes.funnel_rollouts(n_rollouts=12)
    cls, first = _against_oracle(sc)
    print("funnel: %d match, %d switches (parting at %s), %d flagged" % (
        cls.count("match"), cls.count("switch"), first, cls.count("flagged")))
    assert cls.count("flagged") <= 1


def test_studies_run_and_report():
    r = studies.robustness(levels=(0.0, 0.1), trials=64)
    assert r["obstacles"]["success_rate"][0] == 1.0 and r["actuation"]["success_rate"][0] == 1.0
    assert all(0.0 <= v <= 1.0 for k in ("obstacles", "actuation") for v in r[k]["success_rate"])
    f = studies.funnel(ks=(3, 5), n_rollouts=20)
    assert len(f["ratio"]) == 4 and all(v >= 1.0 for d in f["ratio"] for v in d.values())
    print("robustness:", {k: r[k]["success_rate"] for k in ("obstacles", "actuation")}, "funnel:", f["ratio"])
