"""Host-side logic of the serving loop (no device): the admission policy, the
memory accounting and the request stream."""
import numpy as np

from paper_2406_18109_gb300 import serve
from synth import inputs


def _reqs(spec):
    return [{"rid": i, "arrival": t, "kind": k, "size": s, "seed": i} for i, (t, k, s) in enumerate(spec)]


def _need(req, admitted):
    return serve.request_bytes(req["kind"], req["size"])


def test_admit_is_fifo_and_waits_for_arrival():
    q = _reqs([(0.0, "cg", 4), (0.5, "bs", 100), (1.0, "cg", 4)])
    adm, add = serve.admit(q, 0.6, 0, 10 ** 9, {}, 8, _need)
    assert [r["rid"] for r in adm] == [0, 1]
    assert add == serve.request_bytes("cg", 4) + serve.request_bytes("bs", 100)
    adm, _ = serve.admit(q, -1.0, 0, 10 ** 9, {}, 8, _need)
    assert adm == []


def test_admit_respects_budget_without_overtaking():
    q = _reqs([(0.0, "bicgstab", 10), (0.0, "bs", 10)])
    big = serve.request_bytes("bicgstab", 10)
    adm, _ = serve.admit(q, 1.0, 0, big - 1, {}, 8, _need)
    assert adm == []                         # the small request behind it waits too
    adm, _ = serve.admit(q, 1.0, 0, big - 1, {}, 8, _need, evictable=1)
    assert [r["rid"] for r in adm] == [0]    # idle operators can make room
    adm, _ = serve.admit(q, 1.0, 5, big + 400, {}, 8, _need)
    assert [r["rid"] for r in adm] == [0, 1]


def test_admit_slot_limit_per_solver_kind():
    q = _reqs([(0.0, "cg", 4)] * 3 + [(0.0, "bs", 8)])
    adm, _ = serve.admit(q, 1.0, 0, 10 ** 12, {"cg": 1}, 2, _need)
    assert [r["rid"] for r in adm] == [0]    # one free CG slot; FIFO stops there


def test_operator_counted_once_per_new_size():
    srv = serve.Server.__new__(serve.Server)
    srv.ops = {}
    q = _reqs([(0.0, "cg", 6), (0.0, "bicgstab", 6), (0.0, "cg", 8)])
    adm, add = serve.admit(q, 1.0, 0, 10 ** 12, {}, 8, srv._need)
    want = (serve.request_bytes("cg", 6) + serve.request_bytes("bicgstab", 6) + serve.request_bytes("cg", 8)
            + serve.operator_bytes(6) + serve.operator_bytes(8))
    assert len(adm) == 3 and add == want


def test_operator_bytes_matches_the_matrix():
    for m in (3, 5, 8):
        rp, col, val = inputs.poisson3d_csr(m)
        assert serve.operator_bytes(m) == rp.nbytes + col.nbytes + val.nbytes


def test_request_stream_shape():
    r = inputs.serving_requests(3000, seed=3)
    assert [x["rid"] for x in r] == list(range(3000))
    t = np.array([x["arrival"] for x in r])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    assert abs(np.diff(t).mean() - 2e-3) < 0.15e-3       # exponential gaps, mean 2 ms
    kinds = [x["kind"] for x in r]
    for k in serve.KINDS:
        assert abs(kinds.count(k) / 3000 - 1 / 3) < 0.04
    for x in r:
        if x["kind"] == "bs":
            assert 2 ** 16 <= x["size"] <= 2 ** 24
        else:
            assert x["size"] in inputs.SERVE_LADDER
    assert inputs.serving_requests(50, seed=3) == inputs.serving_requests(50, seed=3)


def test_tick_clock_and_summary():
    c = serve.TickClock(0.5)
    c.advance(0.0)
    c.advance(2.0)
    assert c() == 2.5
    res = [serve.Result(i, "cg", 4, arrival=0.0, done=(i + 1) / 100.0, iterations=8) for i in range(100)]
    s = serve.summarize(res, wall_s=2.0)
    assert s["requests"] == 100 and s["sustained_rps"] == 50.0
    assert abs(s["p50_ms"] - 505.0) < 1e-9 and abs(s["p99_ms"] - 990.1) < 1e-9
    assert s["cg"]["count"] == 100 and s["unconverged"] == 0


def test_result_buffers_are_reused_only_when_outputs_are_not_kept(monkeypatch):
    """Page-locked result buffers come from a pool keyed by dtype and a
    power-of-two capacity; a buffer goes back to it after its result is handed
    over, and never when the caller keeps the outputs."""
    made = []

    def fake_host_empty(shape, dtype):
        a = np.empty(shape, dtype)
        made.append(a)
        return a
    monkeypatch.setattr(serve.A.Runtime, "host_empty", staticmethod(fake_host_empty))
    for keep in (False, True):
        made.clear()
        srv = serve.Server(None, None, keep_outputs=keep)
        a = srv._out_buffer(100, np.float64)
        assert len(a) == 128
        srv._recycle(a)
        b = srv._out_buffer(70, np.float64)              # same capacity class (65..128)
        c = srv._out_buffer(100, np.float32)             # another dtype: a new buffer
        srv._recycle(b)
        d = srv._out_buffer(129, np.float64)             # the next class: a new buffer
        assert (b is a) == (not keep)
        assert len(d) == 256 and c is not a and d is not a
        assert len(made) == (3 if not keep else 4)
        assert srv.stats_pool == {"allocated": len(made), "reused": 1 if not keep else 0}
    assert len(serve.Server(None, None)._out_buffer(1, np.float64)) == 1
