"""Serving loop (vine_server_*): each request's result is the same served
alone, served in a mix with other requests, and computed by a batch of its
own; admission by free slots; malformed requests are refused."""
import time

import numpy as np
import pytest

from paper_2509_15180_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2509_15180_gb300 import vine  # noqa: E402

KEYS = ("theta", "l", "tip", "N", "status", "iters")


def _requests(k, replicate=0):
    rng = np.random.default_rng(100 + replicate)
    out = []
    for j in range(k):
        n = int(rng.integers(1, 9))
        out.append(scenes.uneven_batch(n, replicate=700 + 31 * replicate + j, n_range=(20, 60)))
    return out


def _batch_result(sc):
    p = vine.vine_params_default()
    p.threads_per_robot = 32  # the servers below hold at most 64 links per slot: one warp per robot
    b = vine.Batch(sc, p)
    b.simulate()
    st = b.state()
    b.close()
    return dict(theta=st["theta"], l=st["l"], tip=st["tip"], N=st["N"], status=st["status"], iters=st["iters"])


def _wait(srv, rid, limit_s=120.0):
    t0 = time.time()
    while time.time() - t0 < limit_s:
        r = srv.poll(rid, timeout_us=200000)
        if r is not None:
            return r
    raise AssertionError("request %d not finished within %.0f s" % (rid, limit_s))


def _same(a, b, what):
    for k in KEYS:
        assert np.array_equal(np.asarray(a[k]).reshape(-1), np.asarray(b[k]).reshape(-1)), (what, k)


def test_results_same_alone_in_mix_and_batched():
    reqs = _requests(6)
    ref = [_batch_result(sc) for sc in reqs]
    srv = vine.Server(steps_per_tick=3, max_slots=512, max_links=64, max_obs=200, max_act=8, max_request=16)
    alone = []
    for sc in reqs:
        rid = srv.submit(sc)
        assert rid is not None
        alone.append(_wait(srv, rid))
    # the same requests submitted together, interleaved with other traffic
    filler = _requests(6, replicate=1)
    ids = []
    for sc, f in zip(reqs, filler):
        ids.append(srv.submit(sc))
        srv.submit(f)
        time.sleep(0.002)  # arrive while earlier ones are on the GPU
    assert all(i is not None for i in ids)
    mix = [_wait(srv, i) for i in ids]
    st = srv.stats()
    print("served: %d requests in %d ticks, %d robot-link-steps" % (st["requests_done"], st["ticks"],
                                                                   st["robot_link_steps"]))
    for j in range(len(reqs)):
        _same(alone[j], ref[j], "alone vs batch, request %d" % j)
        _same(mix[j], ref[j], "mix vs batch, request %d" % j)
        assert mix[j]["rls"] == alone[j]["rls"]
        assert mix[j]["t_submit"] <= mix[j]["t_admit"] <= mix[j]["t_done"]
    srv.close()


def test_served_configuration_same_alone_in_mix_and_batched():
    """The configuration the benchmark serves: 320-link slots (four-warp
    teams), 200 obstacles, 8 actuators, requests of up to 256 robots grown to
    completion in one launch, four launch lanes; requests drawn like the
    serving workload (links U{20..300}, 5-200 obstacles).  Each result is
    bitwise the same served alone, in a mix that arrives while others are on
    the GPU, and by a batch of its own with the same team size."""
    rng = np.random.default_rng(321)
    reqs = [scenes.uneven_batch(int(rng.integers(1, 7)), replicate=1200 + j, n_range=(20, 300)) for j in range(5)]
    filler = [scenes.uneven_batch(int(rng.integers(4, 24)), replicate=1300 + j, n_range=(20, 300)) for j in range(5)]
    p = vine.vine_params_default()
    p.threads_per_robot = 128  # what the server takes for 320-link slots
    ref = []
    for sc in reqs:
        b = vine.Batch(sc, p)
        b.simulate()
        st = b.state()
        b.close()
        ref.append(dict(theta=st["theta"], l=st["l"], tip=st["tip"], N=st["N"], status=st["status"], iters=st["iters"]))
    srv = vine.Server(max_slots=4096, max_links=320, max_obs=200, max_act=8, max_request=256, lanes=4)
    alone = []
    for sc in reqs:
        rid = srv.submit(sc)
        assert rid is not None
        alone.append(_wait(srv, rid))
    ids = []
    for sc, f in zip(reqs, filler):
        assert srv.submit(f) is not None
        time.sleep(0.003)  # the filler is on the GPU when the request arrives
        ids.append(srv.submit(sc))
    assert all(i is not None for i in ids)
    mix = [_wait(srv, i) for i in ids]
    for j in range(len(reqs)):
        _same(alone[j], ref[j], "alone vs batch, request %d" % j)
        _same(mix[j], ref[j], "mix vs batch, request %d" % j)
        assert mix[j]["rls"] == alone[j]["rls"]
    st = srv.stats()
    print("served configuration: %d requests, %d launches" % (st["requests_done"], st["ticks"]))
    srv.close()


def test_admission_by_free_slots():
    srv = vine.Server(max_slots=8, max_request=8, max_links=64, max_obs=200, max_act=8, steps_per_tick=2)
    big = scenes.uneven_batch(6, replicate=900, n_range=(50, 60))
    r1 = srv.submit(big)
    assert r1 is not None
    assert srv.submit(scenes.uneven_batch(6, replicate=901, n_range=(20, 30))) is None  # 6 + 6 > 8 slots: busy
    r_small = srv.submit(scenes.uneven_batch(2, replicate=902, n_range=(20, 30)))
    assert r_small is not None  # 6 + 2 fit
    assert srv.stats()["free_slots"] == 0
    _wait(srv, r1)
    _wait(srv, r_small)
    assert srv.stats()["free_slots"] == 8
    assert srv.submit(scenes.uneven_batch(6, replicate=901, n_range=(20, 30))) is not None
    srv.close()


def test_refuses_malformed_requests():
    srv = vine.Server(max_slots=64, max_request=4, max_links=40, max_obs=200, max_act=8)
    with pytest.raises(vine.VineError) as e:
        srv.submit(scenes.uneven_batch(5, replicate=903, n_range=(20, 30)))  # more robots than max_request
    assert e.value.status == vine.VINE_EINVAL
    with pytest.raises(vine.VineError) as e:
        srv.submit(scenes.uneven_batch(2, replicate=904, n_range=(41, 50)))  # links beyond the slot capacity
    assert e.value.status == vine.VINE_EINVAL
    sc = scenes.uneven_batch(2, replicate=905, n_range=(20, 30))
    sc["radius"] = sc["radius"].copy()
    sc["radius"][1] = np.nan  # invalid value: that robot only is flagged
    r = _wait(srv, srv.submit(sc))
    assert r["status"][1] == vine.INST_BADINPUT and r["N"][1] == 0
    assert r["N"][0] == sc["n_links"][0]
    with pytest.raises(vine.VineError) as e:
        srv.poll(123456789)
    assert e.value.status == vine.VINE_EINVAL
    srv.close()


def test_poll_timeout_then_result():
    srv = vine.Server(max_slots=256, max_request=64, max_links=320, steps_per_tick=4)
    sc = scenes.uneven_batch(64, replicate=906, n_range=(200, 300))
    rid = srv.submit(sc)
    assert srv.poll(rid, timeout_us=0) is None  # 64 robots x 200-300 links are not done at once
    r = _wait(srv, rid, limit_s=300.0)
    assert np.all((r["N"] == sc["n_links"]) | (r["status"] != 0))
    srv.close()


def _with_cells(sc, cells):
    """The scene with every actuator's cell length drawn from `cells` in turn."""
    sc = dict(sc)
    n = sc["act_l0"].size
    sc["act_l0"] = np.asarray([cells[a % len(cells)] for a in range(n)], np.float32)
    return sc


def test_table_entries_are_reused_after_requests_finish():
    """Table entries are held per live request: a request whose cell lengths
    would exceed max_tables together with the live ones is refused with
    EBUSY, then admitted when the holders finish; over the server's lifetime
    many more distinct cell lengths than max_tables pass through, and every
    result is bitwise the one of a batch of its own (the reused entries are
    rebuilt for their new cell lengths)."""
    srv = vine.Server(max_slots=64, max_request=8, max_links=64, max_obs=200, max_act=8, max_tables=2)
    p = vine.vine_params_default()
    p.threads_per_robot = 32
    base = [scenes.uneven_batch(4, replicate=1400 + k, n_range=(20, 40)) for k in range(6)]
    reqs = [_with_cells(sc, [0.020 + 0.001 * k]) for k, sc in enumerate(base)]  # one new cell length each
    assert all(np.diff(sc["act_ptr"])[:].sum() > 0 for sc in reqs)
    with pytest.raises(vine.VineError) as e:
        srv.submit(_with_cells(base[0], [0.03, 0.031, 0.032]))  # three cell lengths in one request
    assert e.value.status == vine.VINE_EINVAL
    r0 = srv.submit(reqs[0])
    r1 = srv.submit(reqs[1])
    assert r0 is not None and r1 is not None
    assert srv.submit(reqs[2]) is None  # a third live cell length: busy
    out = {0: _wait(srv, r0), 1: _wait(srv, r1)}
    for k in range(2, 6):
        rid = srv.submit(reqs[k])
        assert rid is not None
        out[k] = _wait(srv, rid)
    for k, sc in enumerate(reqs):
        b = vine.Batch(sc, p)
        b.simulate()
        st = b.state()
        b.close()
        ref = dict(theta=st["theta"], l=st["l"], tip=st["tip"], N=st["N"], status=st["status"], iters=st["iters"])
        _same(out[k], ref, "request %d" % k)
    srv.close()
