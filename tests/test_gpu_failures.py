"""Failure detection without any GPU fault: a build cancelled by its host
time limit (the kernels read the error word and stop), and device allocation
failures injected on the host at every allocation of a build.  The library
stays usable afterwards and keeps producing the oracle's structures."""
import time

import numpy as np
import pytest

from paper_1910_06416_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1910_06416_gb300 import build
    build.build()
    import paper_1910_06416_gb300.recsplit as rs
    rs.lib()
    return rs


def test_time_limit_cancels_a_long_build(rs, orc):
    keys = torch.from_numpy(inputs.u64_keys(300_000, 2).view(np.int64)).cuda()  # ~0.3 s at l=16, b=2000
    # load the l = 16 kernels first (their first launch loads them, which blocks the host)
    rs.recsplit_free(rs.recsplit_build_u64(keys[:3000], 16, 2000))
    rs.recsplit_set_timeout_ms(20)
    try:
        t0 = time.time()
        with pytest.raises(rs.RecSplitError) as e:
            rs.recsplit_build_u64(keys, 16, 2000)
        assert e.value.code == rs.E_TIMEOUT
        assert time.time() - t0 < 0.25
    finally:
        rs.recsplit_set_timeout_ms(0)
    small = inputs.u64_keys(20000, 3)
    s = rs.Structure.build_u64(small, 8, 100)
    assert np.array_equal(s.serialize(), orc.build_u64(small, 8, 100))


def test_generous_time_limit_changes_nothing(rs, orc):
    small = inputs.u64_keys(50000, 4)
    rs.recsplit_set_timeout_ms(60_000)
    try:
        s = rs.Structure.build_u64(small, 5, 5)
    finally:
        rs.recsplit_set_timeout_ms(0)
    assert np.array_equal(s.serialize(), orc.build_u64(small, 5, 5))


def test_injected_allocation_failures(rs, orc):
    keys = inputs.u64_keys(20000, 5)
    ref = orc.build_u64(keys, 8, 100)
    failures = 0
    for after in range(0, 60):
        rs.recsplit_inject_alloc_failure(after)
        try:
            s = rs.Structure.build_u64(keys, 8, 100)  # host keys: staging allocation too
            assert np.array_equal(s.serialize(), ref)
            break
        except rs.RecSplitError as err:
            assert err.code == rs.E_NOMEM
            failures += 1
        finally:
            rs.recsplit_inject_alloc_failure(-1)
    assert failures >= 10  # every allocation of the build failed once
    out = np.zeros(keys.shape[0], dtype=np.uint64)
    s = rs.Structure.build_u64(keys, 8, 100)
    rs.recsplit_inject_alloc_failure(0)
    try:
        with pytest.raises(rs.RecSplitError) as e:
            s.lookup_u64(keys, out)  # host buffers need staging
        assert e.value.code == rs.E_NOMEM
    finally:
        rs.recsplit_inject_alloc_failure(-1)
    s.lookup_u64(keys, out)
    assert np.array_equal(out, orc.lookup_u64(ref, keys))
