"""Host checks of the stored oracle results (tests/golden/*_oracle.json)
against the seeded input generators they were written from, and of the DRAM
traffic figure the benchmark reads from the committed ncu summary.  A change
to a generator, or a stored file that no longer matches it, fails here on
the CPU before any GPU parity test compares against a stale file."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1505_01998_gb300 import datagen  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_batch_golden_covers_the_stated_datasets():
    """Every dataset with n <= 16,384 of datagen.batch(512, seed=4) and the
    16 smallest above, each with the size the generator gives it."""
    gold = _load("batch512_oracle.json")
    sizes = datagen.batch_sizes(gold["count"], gold["seed"])
    small = {i for i, n in enumerate(sizes) if n <= 16384}
    above = {i for _, i in sorted((int(n), i) for i, n in enumerate(sizes) if n > 16384)[:16]}
    cases = gold["cases"]
    assert {c["i"] for c in cases} == small | above
    for c in cases:
        assert c["n"] == int(sizes[c["i"]])
        assert 0 <= c["argmin"] < gold["n_h"] and c["argmin"] in c["idx"]
        assert len(c["g"]) == len(c["s_kk"]) == len(c["s_k"]) == len(c["idx"])
        # the stored minimum is the smallest stored value of g
        assert c["g"][c["idx"].index(c["argmin"])] == min(c["g"])


def test_batch_golden_small_dataset_recomputed():
    """The smallest stored dataset recomputed by the oracle from the
    generator's samples equals the stored values exactly (same inputs, same
    fixed-order FP64 arithmetic)."""
    gold = _load("batch512_oracle.json")
    c = min(gold["cases"], key=lambda c: c["n"])
    sets = datagen.batch(gold["count"], seed=gold["seed"])
    x = sets[c["i"]].astype(np.float64)
    assert x.shape == (1, c["n"])
    h = oracle.grid_default(c["n"], 1, gold["n_h"])
    r = oracle.lscv_h(x, h)
    assert int(r["argmin"]) == c["argmin"]
    assert [float(r["g"][k]) for k in c["idx"]] == c["g"]
    p = oracle.plugin(x[0])
    assert float(p["h"]) == c["plugin"]["h"]


@pytest.mark.parametrize("name,n", [("skewed65536_oracle.json", 65536), ("mixture16384_oracle.json", 16384)])
def test_full_golden_grids_are_the_default_grids(name, n):
    gold = _load(name)
    assert gold["n"] == n
    if "cases" in gold:
        for d, case in gold["cases"].items():
            assert np.array_equal(np.asarray(case["h"]), oracle.grid_default(n, int(d), gold["n_h"]))
            assert case["seed"] == 3 + int(d)
    else:
        assert np.array_equal(np.asarray(gold["h"]), oracle.grid_default(n, 1, len(gold["h"])))


def test_benchmark_reads_the_traffic_of_the_current_kernel():
    """bench.py reports the DRAM bytes of the LSCV launch from the committed
    ncu summary only while that summary names the current lscv.cu."""
    import hashlib
    import re
    import bench
    text = open(os.path.join(ROOT, "profiles", "k_lscv_skewed_column.md")).read()
    want = re.search(r"sha256 prefix\s+`([0-9a-f]{16})`", text).group(1)
    have = hashlib.sha256(open(os.path.join(ROOT, "paper_1505_01998_gb300", "csrc", "lscv.cu"),
                                "rb").read()).hexdigest()[:16]
    traffic = bench.profiled_lscv_traffic()
    if want == have:
        assert isinstance(traffic, int) and traffic > 0
    else:
        assert traffic is None
