"""The serving loop: every request's result equals the oracle's sort of the
request and the same request sorted alone, requests overlap on the device,
and admission respects the budget."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import assert_bit_exact, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2603_08929_gb300 import build as b
    b.build()
    torch.cuda.set_device(0)


def request_mix(count, seed):
    rng = np.random.default_rng(seed)
    dts = rng.choice(["int16", "int32", "float32", "float64"], size=count, p=[0.25, 0.35, 0.3, 0.1])
    sizes = np.floor(2.0 ** (10 + 10 * rng.random(count))).astype(np.int64)
    reqs = []
    for i, (dt, n) in enumerate(zip(dts, sizes)):
        # the served workload's value mixes, plus the float edge values (+-0,
        # subnormals, infinities, NaN payloads of both signs) and tie-heavy ints
        if i % 3 == 2:
            dist = "float_edge" if dt.startswith("float") else "zipf"
        else:
            dist = "normal01" if i % 3 else "uniform"
        reqs.append((W.make(dist, dt, int(n), seed=seed * 1000 + i), bool(i % 4 == 0)))
    return reqs


def test_same_alone_and_in_the_mix():
    import torch
    import paper_2603_08929_gb300 as bs
    reqs = request_mix(120, 1)
    alone = []
    for x, desc in reqs:  # each request alone, plain sort
        t = to_device(x)
        bs.bsort_keys(t, descending=desc)
        alone.append(t.cpu().numpy())
    torch.cuda.synchronize()
    srv = bs.Server(num_slots=6, max_request_keys=1 << 20, max_batch=4, batch_keys=1 << 14)
    bufs = [to_device(x) for x, _ in reqs]
    torch.cuda.synchronize()
    srv.pause(True)  # queue everything first so that batching and overlap are deterministic
    for i, (b, (_, desc)) in enumerate(zip(bufs, reqs)):
        srv.submit(b, descending=desc, tag=i)
    assert srv.stats()["pending"] == len(reqs)
    srv.pause(False)
    srv.drain(120)
    done = srv.poll()
    assert sorted(c["tag"] for c in done) == list(range(len(reqs)))
    assert all(c["status"] == 0 for c in done)
    for c in done:
        assert c["t_submit_ns"] <= c["t_admit_ns"] <= c["t_done_ns"]
    for i, b in enumerate(bufs):
        x, desc = reqs[i]
        got = b.cpu().numpy()
        assert_bit_exact(got, O.bsort(x, descending=desc), "request %d (%s) against the oracle" % (i, x.dtype))
        assert_bit_exact(got, alone[i], "request %d: in the mix against alone" % i)
    st = srv.stats()
    assert st["max_concurrent_slots"] > 1  # requests overlapped on the device
    assert st["batches"] < len(reqs)       # small requests shared slots
    srv.close()


def test_budget_limits_requests_in_flight():
    import torch
    import paper_2603_08929_gb300 as bs
    n = 1 << 20
    ws = bs.workspace_bytes(n, "int32")
    budget = 2 * (4 * n + ws) + 1  # room for two such requests
    srv = bs.Server(num_slots=8, hbm_budget_bytes=budget, max_request_keys=n, max_batch=1)
    xs = [W.make("uniform", "int32", n, seed=50 + i) for i in range(8)]
    bufs = [to_device(x) for x in xs]
    torch.cuda.synchronize()
    for i, b in enumerate(bufs):
        srv.submit(b, tag=i)
    srv.drain(60)
    assert len(srv.poll()) == 8
    st = srv.stats()
    assert st["peak_in_flight_bytes"] <= budget
    assert st["max_concurrent_slots"] <= 2
    for x, b in zip(xs, bufs):
        assert_bit_exact(b.cpu().numpy(), O.bsort(x), "budgeted request")
    with pytest.raises(bs.BsortError):
        srv.submit(to_device(np.zeros(n + 1, np.int32)))  # beyond max_request_keys
    srv.close()


def test_two_lanes_share_the_load():
    """Two lanes on this one GPU (the device listed twice): requests go to
    the less loaded lane of their device, both lanes sort, each lane keeps
    its own budget, and every result equals the oracle's."""
    import torch
    import paper_2603_08929_gb300 as bs
    reqs = request_mix(80, 2)
    budget = 48 << 20
    srv = bs.Server(num_slots=2, hbm_budget_bytes=budget, max_request_keys=1 << 20, max_batch=4,
                    batch_keys=1 << 16, devices=[0, 0])
    assert srv.stats()["num_lanes"] == 2
    assert srv.pick_device() == 0
    bufs = [to_device(x) for x, _ in reqs]
    torch.cuda.synchronize()
    srv.pause(True)  # all queued first: the dispatch then depends on queued bytes only
    for i, (b, (_, desc)) in enumerate(zip(bufs, reqs)):
        srv.submit(b, descending=desc, tag=i)
    lanes = [srv.lane_stats(0), srv.lane_stats(1)]
    assert all(ln["queued_bytes"] > 0 for ln in lanes), lanes
    srv.pause(False)
    srv.drain(120)
    done = srv.poll()
    assert sorted(c["tag"] for c in done) == list(range(len(reqs)))
    assert all(c["status"] == 0 for c in done)
    assert {c["lane"] for c in done} == {0, 1}
    for ln in (srv.lane_stats(0), srv.lane_stats(1)):
        assert ln["completed"] > 0 and ln["queued_bytes"] == 0 and ln["in_flight_bytes"] == 0
        assert ln["device"] == 0 and ln["budget_bytes"] == budget
    for i, b in enumerate(bufs):
        x, desc = reqs[i]
        assert_bit_exact(b.cpu().numpy(), O.bsort(x, descending=desc), "request %d (%s)" % (i, x.dtype))
    srv.close()


def test_grouped_requests_take_one_segmented_sort():
    """Small requests of one dtype and direction admitted together share one
    segmented sort: fewer launches than one plain sort each, same bytes."""
    import torch
    import paper_2603_08929_gb300 as bs
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(48):
        dt = ["int32", "float32", "float64", "uint64"][i % 4]
        n = int(2 ** (10 + 6 * rng.random()))
        reqs.append((W.make("float_edge" if dt.startswith("float") else "uniform", dt, n, seed=700 + i), i % 8 == 0))

    def serve(max_batch):
        srv = bs.Server(num_slots=2, max_request_keys=1 << 20, max_batch=max_batch, batch_keys=1 << 18)
        bufs = [to_device(x) for x, _ in reqs]
        torch.cuda.synchronize()
        srv.pause(True)
        for i, (b, (_, desc)) in enumerate(zip(bufs, reqs)):
            srv.submit(b, descending=desc, tag=i)
        srv.pause(False)
        srv.drain(120)
        done = srv.poll()
        assert len(done) == len(reqs) and all(c["status"] == 0 for c in done)
        st = srv.stats()
        srv.close()
        return [b.cpu().numpy() for b in bufs], st

    grouped, st_g = serve(16)
    plain, st_p = serve(1)
    assert st_g["grouped_sorts"] > 0 and st_p["grouped_sorts"] == 0
    assert st_g["launches"] < st_p["launches"] / 2, (st_g["launches"], st_p["launches"])
    for i, (x, desc) in enumerate(reqs):
        want = O.bsort(x, descending=desc)
        assert_bit_exact(grouped[i], want, "grouped request %d" % i)
        assert_bit_exact(plain[i], want, "plain request %d" % i)
