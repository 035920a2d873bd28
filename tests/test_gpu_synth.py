"""Actuator design synthesis (Sec. 4.2) on the GPU against the oracle
(oracle/synth.py): the equilibrium angle of every (pressure, cell length)
pair, the design chosen per target (the rule's integer decision, compared
wherever it is not decided by a difference below the two sides' agreement),
and the chosen designs reproducing their targets in the GPU growth step."""
import numpy as np
import pytest

from oracle import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402

R, PV, LS = 0.03335, 10342.0, 0.025
PRESSURES = np.arange(10e3, 100e3 + 1, 10e3)
L0_MIN, L0_STEP, N_L0 = 0.020, 0.001, 61
TOL = 0.004
AGREE = 1e-8  # rad: the two sides' pair angles agree far better than this


def test_pairs_and_choices_match_oracle():
    rng = np.random.default_rng(12)
    targets = np.concatenate([rng.uniform(0.005, 0.11, 40), [0.0, 0.2, np.nan]])
    g = vine.synthesize(targets, R, PV, LS, PRESSURES, L0_MIN, L0_STEP, N_L0, TOL)
    grid = L0_MIN + L0_STEP * np.arange(N_L0)
    opairs = synth.pair_table(PRESSURES, grid, R, PV, LS)
    err = np.max(np.abs(g["pairs"] - opairs))
    print("pair angles: max |gpu - oracle| = %.3g rad over %d pairs" % (err, opairs.size))
    assert err <= AGREE
    # the choice per target: the oracle's rule on its own pair table, wherever
    # no candidate lies within the two sides' agreement of the tolerance
    # boundary and no two candidates of the highest feasible pressure are
    # that close in deviation (there the decision is unique)
    compared = 0
    for q, t in enumerate(targets):
        if not np.isfinite(t):
            assert g["p_index"][q] == -1 and g["l0_index"][q] == -1 and np.isnan(g["theta_eq"][q])
            continue
        dev = np.abs(opairs - t)
        ip, il = synth.choose(float(t), opairs, PRESSURES, TOL)
        if np.any(np.abs(dev - TOL) <= 2 * AGREE):
            continue
        if ip >= 0:
            d = np.sort(dev[ip][dev[ip] <= TOL])
            if d.size > 1 and d[1] - d[0] <= 2 * AGREE:
                continue
        compared += 1
        assert (g["p_index"][q], g["l0_index"][q]) == (ip, il), (q, t)
        if ip >= 0:
            assert abs(g["theta_eq"][q] - opairs[ip, il]) <= AGREE
        else:
            assert np.isnan(g["theta_eq"][q])
    print("choices compared: %d of %d" % (compared, len(targets)))
    assert compared >= 35
    assert np.mean(g["p_index"][:40] >= 0) >= 0.8


def test_chosen_designs_hold_their_targets_in_the_growth_step():
    targets = np.array([0.02, 0.045, 0.07, 0.095])
    g = vine.synthesize(targets, R, PV, LS, PRESSURES, L0_MIN, L0_STEP, N_L0, TOL)
    n, k = 8, 8
    rows = len(targets)
    sc = dict(n_links=np.full(rows, n, np.int32), l_seg=np.full(rows, LS, np.float32),
              radius=np.full(rows, R, np.float32), pressure=np.full(rows, PV, np.float32),
              base=np.zeros((rows, 3), np.float32), act_ptr=np.arange(rows + 1, dtype=np.int32),
              act_begin=np.zeros(rows, np.float32), act_end=np.full(rows, k, np.float32),
              act_side=np.ones(rows, np.int8),
              act_pressure=PRESSURES[g["p_index"]].astype(np.float32),
              act_l0=(L0_MIN + L0_STEP * g["l0_index"]).astype(np.float32),
              obs_ptr=np.zeros(rows + 1, np.int32), obs_kind=np.zeros(0, np.uint8),
              obs_cx=np.zeros(0, np.float32), obs_cy=np.zeros(0, np.float32),
              obs_a=np.zeros(0, np.float32), obs_b=np.zeros(0, np.float32))
    assert np.all(g["p_index"] >= 0)
    b = vine.Batch(sc)
    b.simulate()
    st = b.state()
    for i, t in enumerate(targets):
        th = b.theta_of(st, i)
        assert st["status"][i] == 0
        assert np.all(np.abs(th - t) <= TOL + 1e-5), (t, th)
    b.close()


def test_invalid_specifications_are_rejected():
    with pytest.raises(vine.VineError):
        vine.synthesize([0.05], R, PV, LS, [-1.0], L0_MIN, L0_STEP, N_L0, TOL)
    with pytest.raises(vine.VineError):
        vine.synthesize([0.05], R, PV, LS, PRESSURES, 0.0, L0_STEP, N_L0, TOL)
    with pytest.raises(vine.VineError):
        vine.synthesize([0.05], R, PV, LS, PRESSURES, L0_MIN, L0_STEP, 0, TOL)


def test_kept_tables_give_bitwise_the_same_synthesis():
    """The second call on a grid copies the FP64 tables the first one built;
    pairs and choices are bitwise those of the first call, and another grid
    (or other sPAM constants) is not served from that grid's tables."""
    targets = np.linspace(0.002, 0.1, 97)
    grid = (0.0205, 0.0007, 23)                      # a grid no other test uses
    a = vine.synthesize(targets, R, PV, LS, PRESSURES, *grid, TOL)
    b = vine.synthesize(targets, R, PV, LS, PRESSURES, *grid, TOL)
    for k in ("pairs", "p_index", "l0_index", "theta_eq"):
        assert np.array_equal(a[k], b[k], equal_nan=(k == "theta_eq")), k
    p = vine.vine_params_default()
    p.a_spam *= 2.0
    c = vine.synthesize(targets, R, PV, LS, PRESSURES, *grid, TOL, params=p)
    assert not np.array_equal(a["pairs"], c["pairs"])
    d = vine.synthesize(targets, R, PV, LS, PRESSURES, grid[0], grid[1], grid[2] - 1, TOL)
    assert np.array_equal(d["pairs"], a["pairs"][:, : grid[2] - 1])
