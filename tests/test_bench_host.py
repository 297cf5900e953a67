"""Host logic of bench.py that needs no GPU.

* The source digest that ties a recorded DRAM-traffic figure to the code it
  was measured on covers a translation unit and exactly the local headers it
  includes (directly or through another header): an edit to such a header
  changes it, an edit to an unrelated header or to a comment does not.
* A recorded figure is returned only while the digest it was taken under
  still matches.
"""
import os

import bench


def _tree(root, files):
    for rel, text in files.items():
        path = os.path.join(root, rel)
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w", encoding="utf-8") as fh:
            fh.write(text)


BASE = {
    "paper_1407_8071_gb300/csrc/k_a.cu": '#include "h1.cuh"\n#include "api.h"\n__global__ void k() {}\n',
    "paper_1407_8071_gb300/csrc/h1.cuh": '#pragma once\n#include "h2.h"\nconstexpr int kOne = 1;\n',
    "paper_1407_8071_gb300/csrc/h2.h": "#pragma once\nconstexpr int kTwo = 2;\n",
    "paper_1407_8071_gb300/csrc/h3.cuh": "#pragma once\nconstexpr int kThree = 3;\n",
    "include/api.h": "#pragma once\nint api(void);\n",
}


def test_digest_follows_includes(tmp_path):
    root = str(tmp_path)
    _tree(root, BASE)
    d0 = bench.source_digest("k_a.cu", root=root)
    # an unrelated header and comments leave it alone
    _tree(root, {"paper_1407_8071_gb300/csrc/h3.cuh": "#pragma once\nconstexpr int kThree = 4;\n"})
    assert bench.source_digest("k_a.cu", root=root) == d0
    _tree(root, {"paper_1407_8071_gb300/csrc/h2.h": "#pragma once\n// a note\nconstexpr int kTwo = 2;  /* two */\n"})
    assert bench.source_digest("k_a.cu", root=root) == d0
    # a header reached through another one, and one under include/, change it
    _tree(root, {"paper_1407_8071_gb300/csrc/h2.h": "#pragma once\nconstexpr int kTwo = 5;\n"})
    d1 = bench.source_digest("k_a.cu", root=root)
    assert d1 != d0
    _tree(root, {"include/api.h": "#pragma once\nint api(int);\n"})
    assert bench.source_digest("k_a.cu", root=root) not in (d0, d1)


def test_recorded_traffic_needs_a_matching_digest(tmp_path, monkeypatch):
    root = str(tmp_path)
    _tree(root, dict(BASE, **{"paper_1407_8071_gb300/csrc/k_filter.cu": '#include "h2.h"\n__global__ void k() {}\n'}))
    monkeypatch.setattr(bench, "ROOT", root)
    d = bench.source_digest()
    _tree(root, {"profiles/dram_traffic.txt": f"# header\nk_x {d} 1234 cmd\nk_y 0000000000000000 99 cmd\n"})
    assert bench.recorded_traffic("k_x") == 1234.0
    assert bench.recorded_traffic("k_y") is None
    _tree(root, {"paper_1407_8071_gb300/csrc/h2.h": "#pragma once\nconstexpr int kTwo = 7;\n"})
    assert bench.recorded_traffic("k_x") is None

