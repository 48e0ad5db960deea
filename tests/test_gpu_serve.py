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
