"""Serving loop: the levels of a multilevel estimate run concurrently (one context
and stream per level) and give bit-identical level records to running them one
after another; requests are independent of the order they are served in."""
import pytest

torch = pytest.importorskip("torch")

from paper_2606_09291_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09291_gb300 import mlsgd
    return mlsgd


CFG = dict(n_levels=3, n0=8, n_modes=64, corr_len=0.3, sigma=1.0, theta=5.0, alpha=1e-4, seed=4, rtol=1e-8,
           max_iter=50, precision="mixed", ir_steps=3, field_tc=1, max_batch=16)
MIX = (16, 8, 2)


@pytest.mark.gpu
def test_concurrent_levels_bitwise_equal(lib):
    from paper_2606_09291_gb300 import serving
    z = torch.tensor(inputs.z_test(32), dtype=torch.float64, device="cuda")
    recs = {}
    for conc in (False, True):
        srv = serving.MixServer(CFG, MIX, concurrent=conc)
        t = srv.serve(2, z, first_request=5)  # requests 5 and 6
        assert len(t) == 2 and all(x > 0 for x in t)
        recs[conc] = [(s.field.clone(), s.scalars.clone()) for s in srv.stats]  # request 6
        srv.close()
    for (f0, s0), (f1, s1) in zip(recs[False], recs[True]):
        assert torch.equal(f0, f1) and torch.equal(s0, s1)
    # request 6 served alone (fresh server) equals request 6 served after request 5
    srv = serving.MixServer(CFG, MIX, concurrent=True)
    srv.serve(1, z, first_request=6)
    for (f0, s0), st in zip(recs[True], srv.stats):
        assert torch.equal(f0, st.field) and torch.equal(s0, st.scalars)
    h = srv.stats[0].host()
    assert h["count"] == MIX[0] and h["noconv"] == 0
    srv.close()


def test_fifo_latency_closed_forms():
    from paper_2606_09291_gb300 import serving
    # arrivals far apart: latency = service time; back to back: the queue builds up
    lat = serving.fifo_latency([10.0] * 5, rate_per_s=0.001)
    assert all(abs(x - 10.0) < 1e-9 for x in lat)
    lat = serving.fifo_latency([10.0] * 50, rate_per_s=1e6)
    assert lat[-1] > 490.0


@pytest.mark.gpu
def test_continuous_batching_same_alone_and_in_mix(lib):
    """Requests of several estimates admitted while others run: each level record
    equals the one computed alone, bit for bit; the requests overlap on the device;
    a tight HBM budget keeps the large requests from running together."""
    from paper_2606_09291_gb300 import serving
    z = torch.tensor(inputs.z_test(32), dtype=torch.float64, device="cuda")
    reqs = serving.poisson_mix_requests(MIX, 3, 0.0, first_estimate=40)  # 9 requests at t = 0
    big = [(l, m) for l, m in enumerate(MIX)]
    srv = serving.ContinuousServer(CFG, 3, big)
    mixed = srv.run(reqs, z, keep=True)
    # overlap on the device's own clock: at least two requests ran at once
    assert serving.device_overlap(mixed)["max_concurrent"] >= 2
    srv.close()
    alone = serving.ContinuousServer(CFG, 1, big)
    for r, req in zip(mixed, reqs):
        one = alone.run([(0.0,) + tuple(req[1:])], z, keep=True)[0]
        assert torch.equal(r["field"], one["field"]) and torch.equal(r["scalars"], one["scalars"])
    alone.close()
    # budget = the largest request's scratch: two level-2 requests never run together
    tight = serving.ContinuousServer(CFG, 3, big)
    tight.set_budget(max(tight.footprint(l, m) for l, m in big))
    res = tight.run(reqs, z)
    l2 = [r for r in res if r["level"] == 2]
    assert len(l2) == 3 and tight.deferred > 0
    for i, a in enumerate(l2):  # device clock: the level-2 requests ran one after another
        for b in l2[i + 1:]:
            assert not (a["dev_start_ms"] < b["dev_end_ms"] and b["dev_start_ms"] < a["dev_end_ms"])
    tight.close()
