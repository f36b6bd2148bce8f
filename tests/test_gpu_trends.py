"""The paper's qualitative claims on the GPU path (Sec. 8): larger leaves give
smaller structures, and construction time grows by about e per unit of leaf
size; bits per key barely depend on the number of keys."""
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


def test_leaf_size_trends(rs):
    keys = torch.from_numpy(inputs.u64_keys(300_000, 4).view(np.int64)).cuda()
    rs.recsplit_set_profiling(True)
    bits, work = {}, {}
    for leaf in range(6, 14):
        h = rs.recsplit_build_u64(keys, leaf, 100)
        bits[leaf] = rs.recsplit_stats(h)["bits_per_key"]
        p = rs.recsplit_last_profile()
        work[leaf] = p["leaf_evals"] + p["split_evals"]
        rs.recsplit_free(h)
    rs.recsplit_set_profiling(False)
    assert all(bits[l + 1] < bits[l] + 0.02 for l in range(6, 13))
    assert bits[13] < bits[6] - 0.2
    # search work per unit of leaf size: about e (the paper plots time)
    ratios = [work[l + 1] / work[l] for l in range(8, 13)]
    assert all(1.8 < r < 4.0 for r in ratios), ratios


def test_bits_per_key_independent_of_n(rs):
    out = []
    for n in (100_000, 1_000_000, 10_000_000):
        h = rs.recsplit_build_u64(torch.from_numpy(inputs.u64_keys(n, 8).view(np.int64)).cuda(), 8, 100)
        out.append(rs.recsplit_stats(h)["bits_per_key"])
        rs.recsplit_free(h)
    assert max(out) - min(out) < 0.03, out


def test_profiling_events_only_and_deterministic_work(rs):
    keys = torch.from_numpy(inputs.u64_keys(200_000, 5).view(np.int64)).cuda()
    rs.recsplit_set_profiling(2)  # phase events, no work-count kernels
    rs.recsplit_free(rs.recsplit_build_u64(keys, 8, 100))
    p = rs.recsplit_last_profile()
    assert p["ms_total"] > 0 and p["leaf_evals"] == 0 and p["split_evals"] == 0
    rs.recsplit_set_profiling(1)
    counts = []
    for _ in range(2):
        rs.recsplit_free(rs.recsplit_build_u64(keys, 8, 100))
        p = rs.recsplit_last_profile()
        counts.append((p["leaf_evals"], p["split_evals"], p["leaf_trials"], p["split_trials"]))
    rs.recsplit_set_profiling(0)
    assert counts[0] == counts[1] and counts[0][0] > 0  # the searches are deterministic


def test_executed_evaluation_counts(rs):
    """The work-counting build also counts the evaluations the searches
    execute, bounded by what the searches must do: every split trial
    evaluates all m keys, rounded up to rounds of 32 indices (with one warp
    per node this count is the same in every build); every leaf index tested
    evaluates at least the first-phase keys (5 of 8) and at most all 8, and a
    leaf tests at most one round (4 x 32 indices) past its first success.
    The leaf count varies a little between builds: which keys of a leaf are
    its first five depends on the order the partition's atomics wrote them
    in, and with it how many indices survive the first phase (the index
    found does not change)."""
    keys = torch.from_numpy(inputs.u64_keys(200_000, 6).view(np.int64)).cuda()
    saved = rs.recsplit_get_tuning(8)
    rs.recsplit_set_tuning(8, {"leaf_warps": 1, "leaf_chunk": 4, "leaf_seeds_per_lane": 4,
                               "split_warps": [1, 1, 1], "leaf_two_phase": 1})
    rs.recsplit_set_profiling(1)
    try:
        profs = []
        for _ in range(2):
            rs.recsplit_free(rs.recsplit_build_u64(keys, 8, 100))
            profs.append(rs.recsplit_last_profile())
    finally:
        rs.recsplit_set_profiling(0)
        rs.recsplit_set_tuning(8, saved)
    p = profs[0]
    assert p["split_evals_executed"] == profs[1]["split_evals_executed"]
    assert abs(p["leaf_evals_executed"] - profs[1]["leaf_evals_executed"]) < 0.01 * p["leaf_evals_executed"]
    max_m = 200  # buckets of b = 100 keys stay far below 200
    assert p["split_evals"] <= p["split_evals_executed"] <= p["split_evals"] + 32 * max_m * p["split_nodes"]
    assert 5 * p["leaf_trials"] <= p["leaf_evals_executed"] <= 8 * (p["leaf_trials"] + 128 * p["leaf_nodes"])
