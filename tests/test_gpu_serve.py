"""The request server: results are the same for a request served alone and
in a mix of concurrent requests of different sizes, and equal the oracle."""

from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2301_10838_gb300 import fields
from paper_2301_10838_gb300.serve import Server

pytestmark = pytest.mark.gpu


def _requests():
    rng = np.random.default_rng(21)
    reqs = []
    for i, side in enumerate([12, 40, 7, 64, 33, 20, 50, 16]):
        shape = (side, side + (i % 3), side + 2 * (i % 2))
        g = fields.grf(shape, -2.5, 5000 + i).astype(np.float32)
        t = float(rng.uniform(-1.0, 1.0))
        reqs.append((torch.from_numpy(np.ascontiguousarray(g)), t))
    return reqs


def test_alone_equals_mix_equals_oracle():
    reqs = _requests()
    srv = Server(hbm_budget_bytes=256 << 20, max_slots=4)
    try:
        alone = []
        for f, t in reqs:
            alone.append(srv.wait(srv.submit(f, t)))
        tickets = [srv.submit(f, t) for f, t in reqs]  # all in flight together
        mix = [srv.wait(tk) for tk in tickets]
    finally:
        srv.close()
    for (f, t), a, m in zip(reqs, alone, mix):
        assert a["npairs"] == m["npairs"] and a["root"] == m["root"]
        assert torch.equal(a["pairs"], m["pairs"])
        assert torch.equal(a["labels"], m["labels"])
        fn = f.numpy()
        p_ref, roots = oracle.pairs(oracle.merge_tree(fn))
        assert np.array_equal(m["pairs"].numpy().view(np.uint32), p_ref)
        assert m["root"] == int(roots[0])
        assert np.array_equal(m["labels"].numpy().view(np.uint32), oracle.components(fn, t))


def test_admission_waits_for_budget():
    """A budget that holds one large request at a time still completes all."""
    reqs = [(torch.from_numpy(fields.white_noise((48, 48, 48), s)), 0.5) for s in range(4)]
    srv = Server(hbm_budget_bytes=4 << 20, max_slots=4)
    try:
        tks = [srv.submit(f, t) for f, t in reqs]
        outs = [srv.wait(tk) for tk in tks]
    finally:
        srv.close()
    for (f, t), o in zip(reqs, outs):
        p_ref, _ = oracle.pairs(oracle.merge_tree(f.numpy()))
        assert np.array_equal(o["pairs"].numpy().view(np.uint32), p_ref)


def test_request_too_large_for_budget_is_refused():
    import paper_2301_10838_gb300 as mt

    srv = Server(hbm_budget_bytes=2 << 20, max_slots=1)
    try:
        with pytest.raises(mt.MtError) as e:
            srv.submit(torch.zeros((64, 64, 64)), 0.0)
        assert e.value.code == -6
    finally:
        srv.close()


@pytest.mark.slow
def test_serve_config_sizes_equal_oracle():
    """Requests drawn from the serving workload (cubic GRF P(k)~k^-2.5, sides
    log-uniform in [32, 384], thresholds U(-2, 2)), including the largest
    sides of the stream, all in flight together: pairs, root and labels of
    each equal the oracle's."""
    stream = fields.serve_stream(200.0, 10.0, 32, 384, seed=11)
    by_side = sorted(stream, key=lambda r: r.side)
    picks = [by_side[-1], by_side[-2], by_side[len(by_side) // 2], by_side[len(by_side) // 4], by_side[0]]
    assert picks[0].side >= 300
    reqs = []
    for r in picks:
        g = fields.grf((r.side, r.side, r.side), -2.5, r.seed, device="cuda").cpu()
        reqs.append((g.contiguous(), r.threshold))
    torch.cuda.empty_cache()
    srv = Server(hbm_budget_bytes=8 << 30, max_slots=4)
    try:
        tickets = [srv.submit(f, t) for f, t in reqs]
        outs = [srv.wait(tk) for tk in tickets]
    finally:
        srv.close()
    for (f, t), o, r in zip(reqs, outs, picks):
        fn = f.numpy()
        p_ref, roots = oracle.pairs(oracle.merge_tree(fn))
        assert o["npairs"] == len(p_ref) and o["root"] == int(roots[0]), r.side
        assert np.array_equal(o["pairs"].numpy().view(np.uint32), p_ref), r.side
        assert np.array_equal(o["labels"].numpy().view(np.uint32), oracle.components(fn, t)), r.side


def test_resident_requery_equals_fresh_request():
    """A keyed request keeps its field and tree on the device; a re-query of
    the key at another threshold (no field sent) gives exactly what a fresh
    one-off request gives, and says it reused the tree."""
    f1 = torch.from_numpy(np.ascontiguousarray(fields.grf((40, 36, 44), -2.5, 77).astype(np.float32)))
    f2 = torch.from_numpy(fields.white_noise((20, 24, 28), 5))
    srv = Server(hbm_budget_bytes=256 << 20, max_slots=4)
    try:
        first = srv.wait(srv.submit_resident(11, f1, -0.3))
        assert not first["reused"]
        again = srv.wait(srv.submit_resident(11, None, 0.4, shape=tuple(f1.shape)))
        fresh = srv.wait(srv.submit(f1, 0.4))
        assert again["reused"] and not fresh["reused"]
        assert again["npairs"] == fresh["npairs"] == first["npairs"] and again["root"] == fresh["root"]
        assert torch.equal(again["pairs"], fresh["pairs"])
        assert torch.equal(again["labels"], fresh["labels"])
        assert srv.resident()[0] == 1
        # a second key; both resident; re-queries in flight together with a build
        tks = [srv.submit_resident(12, f2, 0.5), srv.submit_resident(11, None, 1.0, shape=tuple(f1.shape)),
               srv.submit_resident(12, None, 0.2, shape=tuple(f2.shape))]
        outs = [srv.wait(tk) for tk in tks]
        assert [o["reused"] for o in outs] == [False, True, True]
        for (f, t), o in zip([(f2, 0.5), (f1, 1.0), (f2, 0.2)], outs):
            fn = f.numpy()
            p_ref, roots = oracle.pairs(oracle.merge_tree(fn))
            assert np.array_equal(o["pairs"].numpy().view(np.uint32), p_ref)
            assert np.array_equal(o["labels"].numpy().view(np.uint32), oracle.components(fn, t))
        # a key names one field: another grid under it is refused
        import paper_2301_10838_gb300 as mt

        with pytest.raises(mt.MtError) as e:
            srv.wait(srv.submit_resident(12, f1, 0.0))
        assert e.value.code == -1
        srv.evict(11)
        with pytest.raises(mt.MtError) as e:
            srv.wait(srv.submit_resident(11, None, 0.4, shape=tuple(f1.shape)))
        assert e.value.code == -1
        assert srv.resident()[0] == 1
    finally:
        srv.close()


def _request_bytes(shape):
    import paper_2301_10838_gb300 as mt

    nz, ny, nx = shape
    n = nx * ny * nz
    a = lambda x: (x + 255) & ~255  # noqa: E731
    ws = mt.mt_workspace_bytes(mt.Grid(nx, ny, nz))
    return a(4 * n) + a(8 * n) + a(8 * (n // 2 + 1)) + a(4 * n) + a(ws)


def test_resident_entries_are_evicted_when_room_is_needed():
    big, small = (48, 48, 48), (16, 16, 16)
    budget = _request_bytes(big) + _request_bytes(small) // 2
    srv = Server(hbm_budget_bytes=budget, max_slots=2)
    try:
        fs = torch.from_numpy(fields.white_noise(small, 1))
        srv.wait(srv.submit_resident(1, fs, 0.5))
        assert srv.resident()[0] == 1
        fb = torch.from_numpy(fields.white_noise(big, 2))
        out = srv.wait(srv.submit(fb, 0.5))  # needs the resident entry's memory
        p_ref, _ = oracle.pairs(oracle.merge_tree(fb.numpy()))
        assert np.array_equal(out["pairs"].numpy().view(np.uint32), p_ref)
        assert srv.resident()[0] == 0
    finally:
        srv.close()


def test_large_request_is_not_starved():
    """A large request that cannot run beside any small one is overtaken by at
    most 8 later small requests, then admission waits for it."""
    large, small = (64, 64, 64), (12, 12, 12)
    budget = _request_bytes(large) + _request_bytes(small) // 2
    srv = Server(hbm_budget_bytes=budget, max_slots=4)
    try:
        fl = torch.from_numpy(fields.white_noise(large, 3))
        fsm = [torch.from_numpy(fields.white_noise(small, 100 + i)) for i in range(48)]
        before = [srv.submit(fsm[i], 0.5) for i in range(4)]
        tl = srv.submit(fl, 0.5)
        after = [srv.submit(fsm[i], 0.5) for i in range(4, 48)]
        for tk in before:
            srv.wait(tk)
        rl = srv.wait(tl)
        ra = [srv.wait(tk) for tk in after]
    finally:
        srv.close()
    admitted = lambda r: r["t_submit"] + r["queue_s"]  # noqa: E731
    overtook = sum(1 for r in ra if admitted(r) < admitted(rl))
    assert overtook <= 8, overtook
    assert any(admitted(r) > admitted(rl) for r in ra)  # it did not simply wait until the end
    p_ref, _ = oracle.pairs(oracle.merge_tree(fl.numpy()))
    assert np.array_equal(rl["pairs"].numpy().view(np.uint32), p_ref)
