"""Host-side file formats: G-set style graph files and the hexadecimal
configuration format (no GPU)."""
import numpy as np
import pytest

from paper_2510_21105_gb300 import hexconfig
from paper_2510_21105_gb300 import workloads as wl


@pytest.mark.parametrize("g", [wl.gnp(60, 0.1, seed=3), wl.torus(7, seed=4)], ids=["unsigned", "signed"])
def test_gset_roundtrip(tmp_path, g):
    p = tmp_path / "g.txt"
    wl.write_gset(g, str(p))
    h = wl.read_gset(str(p))
    assert h.n == g.n and h.m == g.m
    assert np.array_equal(h.rp, g.rp) and np.array_equal(h.col, g.col)
    if g.w is None:
        assert h.w is None
    else:
        assert np.array_equal(h.w, g.w)


def test_gset_reads_one_based_text(tmp_path):
    p = tmp_path / "tri.txt"
    p.write_text("4 3\n1 2 1\n2 3 -1\n4 1 1\n")
    g = wl.read_gset(str(p))
    assert g.n == 4 and g.m == 3
    i, j, w = g.edges()
    assert sorted(zip(i.tolist(), j.tolist(), w.tolist())) == [(0, 1, 1), (0, 3, 1), (1, 2, -1)]


@pytest.mark.parametrize("text,err", [("3 1\n1 4 1\n", "out of"), ("3 1\n1 2 2\n", "weights"),
                                      ("3 2\n1 2 1\n", "expected")])
def test_gset_rejects_malformed(tmp_path, text, err):
    p = tmp_path / "bad.txt"
    p.write_text(text)
    with pytest.raises(ValueError, match=err):
        wl.read_gset(str(p))


def test_hex_file_comment_stripping_matches_cli_reader(tmp_path):
    x = np.where(np.arange(37) % 3 == 0, 1, -1).astype(np.int8)
    h = hexconfig.encode(x)
    text = "# best configuration\n" + h[:5] + "\n" + h[5:] + "  # tail\n"
    joined = "".join(line.split("#", 1)[0] for line in text.splitlines(True))
    assert np.array_equal(hexconfig.decode(joined, 37), x)
