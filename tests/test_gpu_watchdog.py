"""The kernels' bounded waits: a wait that can never complete gives up after
its limit and is reported in the context's status word, the context stays
usable, and normal work leaves the word clear.  No fault, trap or hang is
involved: the self-test's barrier simply expects data that never comes."""
import time

import numpy as np
import pytest

from paper_2503_22227_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22227_gb300 import api  # noqa: E402


def test_timed_out_wait_is_reported_and_context_survives():
    ctx = api.Context(W.PRESETS["ckks_n12"])
    keys = ctx.keygen(W.seed_for("watchdog"))
    a = ctx.ct_uniform(W.seed_for("watchdog-in"), 0, 3)
    b = ctx.ct_uniform(W.seed_for("watchdog-in"), 1, 3)
    want = ctx.mul_relin(keys, a, b)
    assert ctx.device_status() == 0          # the inner product's waits all completed
    t0 = time.perf_counter()
    ctx.wait_selftest(20_000_000)            # 20 ms limit
    assert ctx.device_status(clear=False) == 2
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(api.CatfheError) as e:   # catfhe_sync reports it, leaves the word
        ctx.sync()
    assert e.value.code == -8                # ETIMEOUT
    assert ctx.device_status() == 2          # read and clear
    assert ctx.device_status() == 0
    ctx.sync()                               # clear word: OK
    # the context still computes the same result
    assert torch.equal(ctx.mul_relin(keys, a, b), want)
    assert ctx.device_status() == 0
    with pytest.raises(api.CatfheError):
        ctx.wait_selftest(10)                # limit out of range
