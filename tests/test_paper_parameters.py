"""The parameters the paper prints (tests/golden/paper_parameters.txt: iSAX
word and alphabet, Sec. 2; L_max default, Sec. 3.4; EAPCA_TH, SAX_TH and the
leaf size of the experiments, Sec. 4.2) against what the library, the
oracle and the benchmark use.  Host-only: needs no GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "paper_parameters.txt")
HEADER = os.path.join(ROOT, "include", "hercules_gb300.h")


def golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            key, v = line.split()
            vals[key] = float(v)
    return vals


@pytest.fixture(scope="module")
def hk():
    from paper_2212_13297_gb300 import build, binding
    build.build()
    return binding


def test_isax_parameters(hk, oracle_lib):
    g = golden()
    text = open(HEADER).read()
    seg = int(re.search(r"#define HK_ISAX_SEGMENTS (\d+)", text).group(1))
    alpha = int(re.search(r"#define HK_ISAX_ALPHABET (\d+)", text).group(1))
    assert (seg, alpha) == (g["isax_segments"], g["isax_alphabet"])
    import oracle
    assert (oracle.W_PAA, oracle.ALPHABET) == (seg, alpha)
    assert hk.isax_breakpoints().size == alpha - 1


def test_query_defaults(hk):
    g = golden()
    d = hk.query_opts_default()
    assert d["l_max"] == g["l_max_default"]
    assert d["eapca_th"] == pytest.approx(g["eapca_th"], abs=0)
    assert d["sax_th"] == pytest.approx(g["sax_th"], abs=0)
    assert d["flags"] == 0


def test_benchmark_uses_the_papers_leaf_size():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.WORKLOADS["large"]["tau"] == golden()["leaf_size"]
