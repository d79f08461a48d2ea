"""The roofline numerator of bench.py on CPU: the algorithmic bytes of one
relaxation launch, derived here from the per-launch formula of the kernel
table (one color phase: the phase's share of A's CSR, the rows it writes and
the vector block it reads), for the 1024 x 1024 rotated-anisotropy 9-point
workload of the default bench line, plus the invariants of the whole-step
count."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.fixture(scope="module")
def c2():
    mats, color = bench.make_matrix("c2")
    rp, col, _ = mats[0]
    n, nnz = len(rp) - 1, len(col)
    return n, nnz, nnz - n, int(color.max()) + 1


def test_c2_sizes(c2):
    n, nnz, E, ncolors = c2
    # 9-point stencil on 1024^2, neighbours outside the grid dropped: each of
    # the 4 * 1024 boundary rows loses 3 entries, the 4 corners one fewer
    assert n == 1024 * 1024 and nnz == 9 * n - 3 * 4 * 1024 + 4 and E == nnz - n
    assert (n, nnz, E, ncolors) == (1_048_576, 9_424_900, 8_376_324, 2)


def test_relax_launch_bytes_c2_bf16(c2):
    n, nnz, E, C = c2
    K, s_x, s_a = 16, 2, 4
    # one color phase: 1/C of the CSR (column int32 + value), the row starts,
    # its rows written once and the whole vector block read once
    per_launch = (nnz * (4 + s_a) + 4 * (n + 1)) / C + (C + 1) / C * n * K * s_x
    ab = bench.algorithmic_bytes(n, nnz, E, 0, K, 8, C, "bf16", True)
    assert ab["relax_per_launch"] == per_launch == 90_128_402.0


def test_step_bytes_invariants(c2):
    n, nnz, E, C = c2
    E_s = E // 2
    by = {p: bench.algorithmic_bytes(n, nnz, E, E_s, 16, 8, C, p, True)
          for p in ("bf16", "fp32", "fp64")}
    assert by["bf16"]["total"] < by["fp32"]["total"] < by["fp64"]["total"]
    for p, ab in by.items():
        assert ab["relax"] == 8 * ab["sweep"] == 8 * C * ab["relax_per_launch"]
        assert ab["total"] == ab["init"] + ab["relax"] + ab["edge"] + ab["strength"]
        ab16 = bench.algorithmic_bytes(n, nnz, E, E_s, 16, 16, C, p, True)
        assert ab16["relax"] == 2 * ab["relax"]                    # linear in the sweeps
    # the fit pattern of depth d > 1 only adds to the edge pass
    d2 = bench.algorithmic_bytes(n, nnz, E, E_s, 16, 8, C, "bf16", True, nnz_p=3 * nnz)
    assert d2["relax"] == by["bf16"]["relax"] and d2["edge"] > by["bf16"]["edge"]


def test_depth2_pattern_of_c2_operator():
    """The search-depth-2 workload fits over the graph of A^2: on the 9-point
    grid operator that is the 5 x 5 block around each point (25 entries in the
    interior), cut at the boundary; E_2 = 25,104,420 off-diagonals at 1024^2."""
    import oracle
    mats, _ = bench.make_matrix("c6")
    rp, col, _ = mats[0]
    n = len(rp) - 1
    prp, pcol = oracle.distance_graph(rp, col, 2)
    N = 1024
    # rows lose 2 (boundary line) or 1 (next line) of the 5 offsets per direction
    per_axis = [5] * N
    per_axis[0] = per_axis[-1] = 3
    per_axis[1] = per_axis[-2] = 4
    s = sum(per_axis)
    assert len(pcol) == s * s and len(pcol) - n == 25_104_420
    i = 500 * N + 500
    assert prp[i + 1] - prp[i] == 25


def test_recorded_traffic_follows_code_not_comments(tmp_path, monkeypatch):
    """The recorded DRAM bytes of a kernel stay valid through edits of its
    comments and layout, and are dropped once its code changes."""
    src = ("// sweep kernel\n__global__ void k(int *p) { /* one store */ p[0] = 1; }\n"
           "const char *s = \"// not a comment\";\n")
    assert bench._code_only(src) == bench._code_only(src.replace("// sweep kernel", "// renamed note")
                                                     .replace("/* one store */", "")
                                                     .replace("p[0] = 1;", "p[0]  =  1;"))
    assert "// not a comment" in bench._code_only(src)
    assert bench._code_only(src) != bench._code_only(src.replace("p[0] = 1", "p[0] = 2"))
    csrc = tmp_path / "paper_1106_5990_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.source_sha("k.cu")
    table = tmp_path / "traffic.json"
    table.write_text('{"relax/fp32/K16/c2": {"source_sha": "%s", "dram_bytes_per_launch": 123.0}}' % sha)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(table))
    assert bench.recorded_traffic("relax/fp32/K16/c2", sha) == 123.0
    (csrc / "k.cu").write_text(src.replace("// sweep kernel", "// edited note"))
    assert bench.recorded_traffic("relax/fp32/K16/c2", bench.source_sha("k.cu")) == 123.0
    (csrc / "k.cu").write_text(src.replace("p[0] = 1", "p[0] = 3"))
    assert bench.recorded_traffic("relax/fp32/K16/c2", bench.source_sha("k.cu")) is None
