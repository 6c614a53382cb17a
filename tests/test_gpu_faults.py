"""Failure detection without a GPU fault.

* A bounded device wait that runs out: a test-only switch (MPWSD_TEST_TC_STALL,
  read when a code is loaded) makes the tensor-core scoring kernel's producer
  issue no copies, so the MMA issuer waits on a barrier nothing completes. The
  wait gives up after 20 ms, the kernel records an error word, frees its TMEM
  and exits; the host sees MPWSD_ETIMEOUT from mpwsd_sync and the error flag on
  the affected frames, and the context stays usable for other handles.
* An allocation failure injected on the host (MPWSD_TEST_FAIL_ALLOC=k fails
  the k-th device allocation of the process) returns MPWSD_ENOMEM and leaves
  the handle usable.
"""
import multiprocessing as mproc
import os

import numpy as np
import pytest

import synth
from gpu_common import cuda_or_skip, to_words, torch

pytestmark = pytest.mark.gpu


def test_tc_wait_timeout_is_reported_and_context_survives():
    mp = cuda_or_skip()
    wl = synth.make_workload("rm26_crc6", 1.0, 2000, seed=31)
    y = torch.from_numpy(wl.y).cuda()
    os.environ["MPWSD_TEST_TC_STALL"] = "1"
    try:
        stalled = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    finally:
        del os.environ["MPWSD_TEST_TC_STALL"]
    cw, fl = stalled.decode(y, 8, 1, score_mode="bf16x2")
    with pytest.raises(mp.MpwsdError) as ei:
        stalled.sync()
    assert ei.value.status == mp.ETIMEOUT
    flags = fl.cpu().numpy().view(np.uint16)
    stage2 = (flags & mp.FLAG_STAGE2) != 0
    assert stage2.any() and np.all((flags[stage2] & mp.FLAG_ERROR) != 0)
    stalled.sync()  # the error word was cleared by the first report
    # the same context keeps decoding correctly with a normal handle
    good = mp.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    a_cw, a_fl = good.decode(y, 8, 4, score_mode="bf16x2")
    b_cw, b_fl = good.decode(y, 8, 4, score_mode="fp32")
    good.sync()
    assert torch.equal(a_cw, b_cw) and torch.equal(a_fl, b_fl)
    assert np.mean(np.any(to_words(a_cw) != synth.pack_bits(wl.cw), axis=1)) < 0.5


def _alloc_child(q):
    import torch as th

    from paper_2602_08501_gb300 import mpwsd

    out = {}
    # device allocations 1..9: flats table (offsets, pattern indices), pattern bits, supports, tiles, CRC
    # masks, generator rows, OSD row sets, stats
    code = mpwsd.Code.rm(6, 2, crc_poly=0x21, crc_len=6, weights=[16])
    wl = synth.make_workload("rm26_crc6", 1.0, 500, seed=32)
    y = th.from_numpy(wl.y).cuda()
    try:
        code.decode(y, 8, 4)  # allocation 10 (the handle's workspace) fails
        out["first"] = "ok"
    except mpwsd.MpwsdError as e:
        out["first"] = e.status
    cw, fl = code.decode(y, 8, 4)  # allocation 11 succeeds
    code.sync()
    cw2, fl2 = code.decode(y, 8, 4, score_mode="fp32")
    code.sync()
    out["second_equal"] = bool(th.equal(cw, cw2) and th.equal(fl, fl2))
    q.put(out)


def test_injected_allocation_failure_returns_enomem():
    cuda_or_skip()
    ctx = mproc.get_context("spawn")
    q = ctx.Queue()
    env_old = os.environ.get("MPWSD_TEST_FAIL_ALLOC")
    os.environ["MPWSD_TEST_FAIL_ALLOC"] = "10"
    try:
        p = ctx.Process(target=_alloc_child, args=(q,))
        p.start()
        out = q.get(timeout=300)
        p.join(timeout=60)
    finally:
        if env_old is None:
            del os.environ["MPWSD_TEST_FAIL_ALLOC"]
        else:
            os.environ["MPWSD_TEST_FAIL_ALLOC"] = env_old
    assert p.exitcode == 0
    assert out["first"] == -2  # MPWSD_ENOMEM
    assert out["second_equal"]
