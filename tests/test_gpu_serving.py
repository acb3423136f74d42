"""The private-query serving workload on the device: 1000 x 4 encrypted
table at N = 2^16, L = 24 (K = 8 special primes), range predicate through
the degree-63 sign polynomial and a rotate-and-add sum over 1024 slots.

Each request's encrypted answer must be bit-identical whether it ran alone
or interleaved with other requests in continuously batched ticks (the
arithmetic is exact and deterministic), and its decryption must be within
1000 * 2^-20 of the float64 evaluation of the same circuit."""
import copy

import numpy as np
import pytest

from paper_2503_22227_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2503_22227_gb300 import serving as S  # noqa: E402


@pytest.fixture(scope="module")
def table():
    return S.Table(W.PRESETS["ckks_n16_k8"], bound_pairs=4)


def test_results_identical_alone_and_in_the_mix(table):
    reqs = S.make_requests(table, 8, rate=400.0, seed="serve-test")
    eng = S.GpuEngine(table, lanes=4)
    st = S.serve(reqs, eng, budget_bytes=6 * table.need, max_active=4)
    assert st.served == 8 and st.max_active <= 4
    assert st.ticks > len(table.circuit.stages())
    assert st.peak_reserved <= 6 * table.need
    for r in reqs:
        assert r.finished > r.admitted >= r.arrival
    for r in reqs:
        solo = copy.copy(r)
        solo.arrival, solo.result, solo.state = 0.0, None, None
        e1 = S.GpuEngine(table, lanes=1)
        S.serve([solo], e1, budget_bytes=table.need, max_active=1)
        assert torch.equal(solo.result, r.result), r.id


def test_answers_match_the_float_circuit(table):
    reqs = S.make_requests(table, 4, rate=0.0, seed="serve-acc")
    eng = S.GpuEngine(table, lanes=4)
    S.serve(reqs, eng, budget_bytes=8 * table.need, max_active=8)
    for r in reqs:
        got = table.decrypt_answer(r.result)
        want = table.float_answer(r.col_a, r.col_b, r.bounds)
        assert abs(got - want) < 1000 * 2.0 ** -20, (r.id, got, want)
        # and the predicate's own definition, evaluated directly in numpy
        lo, hi = table.bounds[r.bounds]
        a, b = table.values[r.col_a], table.values[r.col_b]
        p = lambda x: np.polynomial.chebyshev.chebval(x, S.sign_coefficients())
        direct = float(np.sum((1 + p(a - lo)) * (1 + p(hi - a)) / 4 * b))
        assert abs(got - direct) < 1000 * 2.0 ** -20, (r.id, got, direct)


def test_admission_by_memory(table):
    reqs = S.make_requests(table, 5, rate=0.0, seed="serve-adm")
    eng = S.GpuEngine(table, lanes=2, keep_results=False)
    st = S.serve(reqs, eng, budget_bytes=2 * table.need + 1, max_active=64)
    assert st.max_active == 2 and st.served == 5
    with pytest.raises(ValueError):
        S.serve(S.make_requests(table, 1, 0.0, "x"), eng, budget_bytes=table.need - 1)


def test_search_and_average(table):
    """Avg(b) where lo <= a <= hi: the circuit's encrypted sum and count, the
    two-party multiply-inverse on the count (the client only sees the count
    times a random mask), one HMult; against the same soft predicate in numpy."""
    res = S.search_and_average(table, 2, 3, 1, rng=np.random.default_rng(11))
    total, count = table.float_avg_parts(2, 3, 1)
    assert abs(res["count"] - count) < 1000 * 2.0 ** -20
    assert abs(res["sum"] - total) < 1000 * 2.0 ** -20
    assert abs(res["avg"] - total / count) < 1e-7
    assert abs(res["masked_count_seen_by_client"] - count) > 1e-3
    # the float circuit itself is the soft predicate up to the scale drift of
    # the prime chain (relative 1e-4)
    lo, hi = table.bounds[1]
    a, b = table.values[2], table.values[3]
    p = lambda x: np.polynomial.chebyshev.chebval(x, S.sign_coefficients())
    mask = (1 + p(a - lo)) * (1 + p(hi - a)) / 4
    assert abs(count - mask.sum()) < 1e-4 * mask.sum()
    assert abs(total / count - (mask * b).sum() / mask.sum()) < 1e-4
