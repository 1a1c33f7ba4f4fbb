"""Failures made on the host, never on the GPU: an allocation that fails
(GLCM_FAULT=alloc makes the library's device allocations report failure
before cudaMalloc is called) and an admission queue that is full.  Each must
come back as its status code, and the library must keep working afterwards.
The device-side bounded waits (the vote kernel's tile mbarrier polls) are
not made to run out here: that needs a copy that never lands, which no
host-side input can cause."""
import numpy as np
import pytest
import torch

import glcm_synth as S
import oracle
import paper_1710_06189_gb300 as G
from conftest import to_u32

pytestmark = pytest.mark.gpu


def test_alloc_fault_in_create_and_in_scratch_then_recovery(monkeypatch):
    img = S.iid(S.BASE_SEED + 61, 300, 700, np.uint8)
    offs = S.CONTENTION_OFFSETS
    want = oracle.glcm(img, 16, offs)
    monkeypatch.setenv("GLCM_FAULT", "alloc")
    with pytest.raises(G.GlcmError) as e:
        G.Context(0)
    assert e.value.status == G.binding.GLCM_ERR_NOMEM
    monkeypatch.delenv("GLCM_FAULT")
    with G.Context(0) as ctx:
        d = torch.from_numpy(img).cuda()
        # A fresh context allocates its tables on first use: make that fail.
        monkeypatch.setenv("GLCM_FAULT", "alloc")
        with pytest.raises(G.GlcmError) as e:
            ctx.compute(d, 16, offs)
        assert e.value.status == G.binding.GLCM_ERR_NOMEM
        monkeypatch.delenv("GLCM_FAULT")
        got = ctx.compute(d, 16, offs)
        torch.cuda.synchronize()
        assert np.array_equal(to_u32(got), want)


def test_full_admission_queue_is_busy_and_recovers():
    """An arena that holds one request (2048^2 uint8 = 4 MiB + counts) and a
    queue of one: submitting faster than requests finish must be refused with
    GLCM_ERR_BUSY, and every accepted request must still be exact."""
    side, offs = 2048, S.CONTENTION_OFFSETS
    imgs = [torch.from_numpy(S.iid(S.BASE_SEED + 70 + k, side, side, np.uint8)).pin_memory() for k in range(4)]
    with G.Server(0, hbm_budget_bytes=6 << 20, lanes=1, max_queue=1) as srv:
        accepted, busy = [], 0
        for attempt in range(400):
            k = attempt % len(imgs)
            try:
                accepted.append((k, srv.submit(imgs[k], 16, offs)))
            except G.GlcmError as e:
                assert e.status == G.GLCM_ERR_BUSY, e
                busy += 1
                if busy >= 3:
                    break
        assert busy >= 1, "a queue of one never filled"
        assert srv.stats()["queue_peak"] <= 1
        for k, t in accepted:
            st, _, (c, _, _) = srv.wait(t)
            assert st == G.GLCM_OK, srv.last_error()
            assert np.array_equal(c.numpy().view(np.uint32), oracle.glcm(imgs[k].numpy(), 16, offs))
        # Once drained, the server admits again.
        st, _, (c, _, _) = srv.wait(srv.submit(imgs[0], 16, offs))
        assert st == G.GLCM_OK
        assert np.array_equal(c.numpy().view(np.uint32), oracle.glcm(imgs[0].numpy(), 16, offs))


def test_measured_ceilings_are_ordered():
    """glcm_measure_ceilings: interleaved copies never conflict, so they are
    at least as fast as random words of one copy; the streaming read rate is
    a plausible HBM rate."""
    c = G.binding.glcm_measure_ceilings(0)
    assert c["sm_count"] > 0
    assert c["red_interleaved_per_s"] > 1e11
    assert c["red_interleaved_per_s"] >= 0.9 * c["red_random_one_copy_per_s"]
    assert c["red_same_word_per_s"] > 1e11
    assert 100.0 < c["hbm_read_gbs"] < 20000.0
