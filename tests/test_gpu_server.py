"""Request server (continuous batching) through the C ABI.

Results decoded in a mix of concurrent requests of several lengths and codes
equal the results of the same requests decoded alone (bit-exact, float32
min-sum), and a sample equals the oracle; admission refusals, the memory
budget and the bounded wait behave as declared.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1204_5882_gb300 import synth as S  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_5882_gb300 import build
    build.build()
    from paper_1204_5882_gb300 import polar
    return polar


def make_requests(P, count, seed, sizes=(10, 12, 14, 16)):
    rng = np.random.default_rng(seed)
    codes = {}
    reqs = []
    for i in range(count):
        n = int(rng.choice(sizes))
        kind = int(rng.integers(0, 3))
        if (n, kind) not in codes:
            if kind == 0:
                fz, _ = O.frozen_set(n, "bsc", 0.03, 0.6)
            elif kind == 1:
                fz, _ = O.frozen_set(n, "biawgn", 1.0, 0.4)
            else:
                fz = (rng.random(1 << n) < 0.5).astype(np.uint8)
            codes[(n, kind)] = (fz, P.polar_frozen_set_from_mask(n, S.pack_bits(fz)))
        fz, fs = codes[(n, kind)]
        F = int(rng.integers(1, 3))
        N = 1 << n
        L = rng.normal(0.7, 2.0, (F, N)).astype(np.float32)
        fvb = (rng.integers(0, 2, (F, N)) * fz).astype(np.uint8)
        fvw = np.stack([S.pack_bits(r) for r in fvb])
        reqs.append(dict(n=n, F=F, fz=fz, fs=fs, L=L, fvb=fvb,
                         llr=torch.from_numpy(L).to(DEV),
                         fv=torch.from_numpy(fvw.view(np.int32)).to(DEV)))
    torch.cuda.synchronize()          # the server's streams do not wait on torch's stream
    return reqs


@pytest.mark.gpu
@pytest.mark.parametrize("persistent,prec", [(False, "fp32"), (True, "fp32"), (True, "fp16"),
                                             (True, "int8")])
def test_results_identical_alone_and_in_mix(P, persistent, prec):
    """A request decoded in the mix equals the same request decoded alone.
    Reduced storage rounds the levels above the subtree size, so the lone
    decodes use the persistent server's subtree size ("persist_log2")."""
    reqs = make_requests(P, 40, 11)
    stream = torch.cuda.Stream()
    alone = []
    saved = {k: P.polar_config_get(k) for k in ("autotune", "subtree_log2")}
    if prec != "fp32":
        P.polar_config_set("autotune", 0)
        P.polar_config_set("subtree_log2", P.polar_config_get("persist_log2"))
    try:
        for r in reqs:                               # one at a time, synchronously
            xh = torch.zeros_like(r["fv"])
            P.polar_sc_decode_many(r["fs"], r["F"], r["llr"], r["fv"], xh, None, "minsum", prec,
                                   stream)
            stream.synchronize()
            alone.append(xh.cpu())
    finally:
        for k, v in saved.items():
            P.polar_config_set(k, v)
    srv = P.Server(max_inflight=16, max_queue=1024, persistent=persistent, max_log2n=16,
                   prec=prec)
    outs, tickets = [], []
    for r in reqs:
        outs.append(torch.full_like(r["fv"], -1))
    torch.cuda.synchronize()                         # outputs initialised before any decode
    for r, xh in zip(reqs, outs):                    # all at once: they overlap
        t = srv.submit(r["fs"], r["F"], r["llr"], r["fv"], xh)
        assert t is not None
        tickets.append(t)
    for t in tickets:
        st, q_ms, lat_ms = srv.wait(t, 60000.0)
        assert st == P.POLAR_OK and lat_ms >= q_ms >= 0.0
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(reqs)
    for r, a, b in zip(reqs, alone, outs):
        assert torch.equal(a, b.cpu())
    if prec != "fp32":
        return
    for r, b in list(zip(reqs, outs))[:6]:           # and the oracle agrees
        got = b.cpu().numpy().view(np.uint32)
        for f in range(r["F"]):
            _, ox = O.sc_decode(r["L"][f], r["fz"], r["fvb"][f], "minsum")
            assert np.array_equal(S.unpack_bits(got[f], 1 << r["n"]), ox)


@pytest.mark.gpu
def test_admission_refused_when_queue_full(P):
    reqs = make_requests(P, 30, 12, sizes=(16,))
    srv = P.Server(max_inflight=1, max_queue=2)
    accepted, refused = [], 0
    outs = [torch.zeros_like(r["fv"]) for r in reqs]
    torch.cuda.synchronize()
    for r, xh in zip(reqs, outs):
        t = srv.submit(r["fs"], r["F"], r["llr"], r["fv"], xh)
        if t is None:
            refused += 1
        else:
            accepted.append(t)
    assert refused > 0 and accepted
    for t in accepted:
        assert srv.wait(t)[0] == P.POLAR_OK
    assert srv.stats()["refused"] == refused
    srv.close()


@pytest.mark.gpu
def test_memory_budget_serialises_and_rejects(P):
    reqs = make_requests(P, 6, 13, sizes=(18,))
    need = max((1 << 18) - (1 << 13), 0) * 4 * 2      # two frames of 2^18 in FP32
    srv = P.Server(max_inflight=8, max_queue=64, mem_budget=need)
    outs = [torch.zeros_like(r["fv"]) for r in reqs]
    torch.cuda.synchronize()
    tickets = [srv.submit(r["fs"], r["F"], r["llr"], r["fv"], xh) for r, xh in zip(reqs, outs)]
    for t in tickets:
        assert srv.wait(t)[0] == P.POLAR_OK
    assert srv.stats()["scratch_bytes"] <= need
    # a request whose scratch alone exceeds the budget fails with ENOMEM
    big = make_requests(P, 1, 14, sizes=(20,))[0]
    xh = torch.zeros_like(big["fv"])
    torch.cuda.synchronize()
    t = srv.submit(big["fs"], big["F"], big["llr"], big["fv"], xh)
    assert srv.wait(t)[0] == P.POLAR_ENOMEM
    srv.close()


@pytest.mark.gpu
def test_bounded_wait_and_bad_tickets(P):
    r = make_requests(P, 1, 15, sizes=(16,))[0]
    srv = P.Server(max_inflight=2)
    xh = torch.zeros_like(r["fv"])
    torch.cuda.synchronize()
    t = srv.submit(r["fs"], r["F"], r["llr"], r["fv"], xh)
    try:
        st = srv.wait(t, 0.0)                        # may already be done
    except P.PolarError as e:                        # still running: bounded wait expired
        assert e.status == P.POLAR_ETIMEDOUT
        st = srv.wait(t, 60000.0)
    assert st[0] == P.POLAR_OK
    with pytest.raises(P.PolarError):
        srv.poll(t)                                  # reported once, then forgotten
    with pytest.raises(P.PolarError):
        srv.poll(987654321)
    srv.close()


# ------------------------------------------------------------------ persistent mode
def alone_results(P, reqs):
    stream = torch.cuda.Stream()
    out = []
    for r in reqs:
        xh = torch.zeros_like(r["fv"])
        P.polar_sc_decode_many(r["fs"], r["F"], r["llr"], r["fv"], xh, None, "minsum", "fp32",
                               stream)
        stream.synchronize()
        out.append(xh.cpu())
    return out


@pytest.mark.gpu
def test_persistent_server_admits_while_running(P):
    """Requests submitted in waves while earlier ones decode join the running
    launch: results equal the alone results, and the server makes far fewer
    launches than requests."""
    import time
    reqs = make_requests(P, 60, 21, sizes=(10, 12, 14, 16, 18))
    alone = alone_results(P, reqs)
    srv = P.Server(max_inflight=64, max_queue=1024, persistent=True, max_log2n=18)
    outs = [torch.full_like(r["fv"], -1) for r in reqs]
    torch.cuda.synchronize()
    before = P.polar_kernel_launches()
    tickets = []
    for w in range(6):                               # six waves, 10 requests each
        for r, xh in list(zip(reqs, outs))[10 * w:10 * w + 10]:
            t = srv.submit(r["fs"], r["F"], r["llr"], r["fv"], xh)
            assert t is not None
            tickets.append(t)
        time.sleep(0.0003)
    for t in tickets:
        st, q_ms, lat_ms = srv.wait(t, 60000.0)
        assert st == P.POLAR_OK and lat_ms >= q_ms >= 0.0
    launches = P.polar_kernel_launches() - before
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(reqs) and stats["launched"] == len(reqs)
    assert 1 <= launches < len(reqs)
    for a, b in zip(alone, outs):
        assert torch.equal(a, b.cpu())


@pytest.mark.gpu
def test_persistent_server_relaunches_after_idle(P):
    """The resident launch ends after a quiet millisecond; a later request
    starts a new one and completes."""
    import time
    reqs = make_requests(P, 3, 22, sizes=(12, 16))
    alone = alone_results(P, reqs)
    srv = P.Server(max_inflight=8, persistent=True, max_log2n=16)
    outs = [torch.full_like(r["fv"], -1) for r in reqs]
    torch.cuda.synchronize()
    before = P.polar_kernel_launches()
    for r, xh in zip(reqs, outs):
        t = srv.submit(r["fs"], r["F"], r["llr"], r["fv"], xh)
        assert srv.wait(t, 60000.0)[0] == P.POLAR_OK
        time.sleep(0.02)                             # well past the idle limit
    assert P.polar_kernel_launches() - before == len(reqs)
    srv.close()
    for a, b in zip(alone, outs):
        assert torch.equal(a, b.cpu())


@pytest.mark.gpu
def test_persistent_server_refuses_long_codes_and_huge_requests(P):
    r = make_requests(P, 1, 23, sizes=(16,))[0]
    srv = P.Server(max_inflight=4, persistent=True, max_log2n=14)
    xh = torch.zeros_like(r["fv"])
    with pytest.raises(P.PolarError) as e:
        srv.submit(r["fs"], r["F"], r["llr"], r["fv"], xh)
    assert e.value.status == P.POLAR_EINVAL
    srv.close()
    with pytest.raises(P.PolarError) as e:             # scratch of one CTA over budget
        P.Server(max_inflight=4, persistent=True, max_log2n=22, mem_budget=1 << 20)
    assert e.value.status == P.POLAR_ENOMEM


# ------------------------------------------------------------------ cancellation
@pytest.mark.gpu
@pytest.mark.parametrize("persistent", [False, True])
def test_cancel_withdraws_only_queued_requests(P, persistent):
    """A withdrawn request reports ECANCELED and its outputs are never
    written; a request that already runs or has finished is not withdrawn and
    completes with the result it has alone.  With one slot, requests queue
    behind the 2^16 decodes ahead of them, so the last one is still queued
    when it is cancelled.  (The persistent ring may take requests at once,
    so there either outcome is possible, and each is checked.)"""
    reqs = make_requests(P, 8, 21, sizes=(16,))
    expect = alone_results(P, reqs)
    srv = P.Server(max_inflight=1, persistent=persistent)
    tickets, outs = [], []
    for r in reqs:
        xh = torch.full_like(r["fv"], -1)
        torch.cuda.synchronize()
        tickets.append(srv.submit(r["fs"], r["F"], r["llr"], r["fv"], xh))
        outs.append(xh)
    withdrawn = [False] * 4 + [srv.cancel(t) for t in tickets[4:]]
    if not persistent:
        assert withdrawn[-1]
    for i, (t, xh) in enumerate(zip(tickets, outs)):
        st = srv.wait(t, 60000.0)
        if withdrawn[i]:
            assert st[0] == P.POLAR_ECANCELED
            assert bool(torch.all(xh == -1))
        else:
            assert st[0] == P.POLAR_OK
            assert torch.equal(xh.cpu(), expect[i])
    with pytest.raises(P.PolarError):
        srv.cancel(tickets[0])                       # reported, so forgotten
    srv.close()
