"""The launch-shape cache of the autotuner (host only: no GPU call is made)."""
import os

import pytest

from paper_1810_01054_gb300 import build as B
from paper_1810_01054_gb300 import mpm


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    mpm.lib()


SHAPES = [(3, 256), (8, 128), (2, 256), (6, 256)]  # p2g, g2p, p2g_adj, adj_gather


def test_store_then_lookup_and_log2_buckets():
    mpm.tune_cache_store(2, 30000, 1024, 152, SHAPES)
    assert mpm.tune_cache_lookup(2, 30000, 1024, 152) == SHAPES
    # the key buckets particles and tiles by floor(log2): 16384..32767 and 1024..2047 share it
    assert mpm.tune_cache_lookup(2, 16384, 2047, 152) == SHAPES
    assert mpm.tune_cache_lookup(2, 32768, 1024, 152) is None
    assert mpm.tune_cache_lookup(2, 30000, 1023, 152) is None
    assert mpm.tune_cache_lookup(3, 30000, 1024, 152) is None
    assert mpm.tune_cache_lookup(2, 30000, 1024, 148) is None


def test_shapes_outside_the_candidates_are_refused():
    bad = [(5, 256), (8, 128), (2, 256), (6, 256)]  # 5 CTAs per SM is not a P2G candidate
    with pytest.raises(mpm.MPMError):
        mpm.tune_cache_store(3, 1000, 64, 152, bad)
    with pytest.raises(mpm.MPMError):  # 128-thread P2G CTAs exist in 2D only
        mpm.tune_cache_store(3, 1000, 64, 152, [(4, 128)] + SHAPES[1:])
    with pytest.raises(mpm.MPMError):  # and only at the listed CTAs per SM
        mpm.tune_cache_store(2, 1000, 64, 152, [(2, 128)] + SHAPES[1:])
    with pytest.raises(mpm.MPMError):  # the adjoint gather's CTA size is not tuned
        mpm.tune_cache_store(2, 1000, 64, 152, SHAPES[:3] + [(4, 128)])
    assert mpm.tune_cache_lookup(3, 1000, 64, 152) is None
    assert mpm.tune_cache_lookup(2, 1000, 64, 152) is None
    mpm.tune_cache_store(2, 1000, 64, 152, [(4, 128), (8, 128), (6, 128), (6, 256)])
    assert mpm.tune_cache_lookup(2, 1000, 64, 152) == [(4, 128), (8, 128), (6, 128), (6, 256)]


def test_file_round_trip(tmp_path):
    mpm.tune_cache_store(3, 1_000_000, 32768, 152, SHAPES)
    f1 = tmp_path / "a.txt"
    mpm.tune_cache_save(str(f1))
    text = f1.read_text().splitlines()
    assert text[0].startswith("gbmpm-tune 1")
    assert "3 19 15 152 3 256 8 128 2 256 6 256" in text
    # a second file written by hand is merged in
    f2 = tmp_path / "b.txt"
    f2.write_text("gbmpm-tune 1\n\n2 10 6 132 2 256 16 128 8 256 2 256\n")
    mpm.tune_cache_load(str(f2))
    assert mpm.tune_cache_lookup(2, 1500, 100, 132) == [(2, 256), (16, 128), (8, 256), (2, 256)]
    # and everything written again reads back the same
    f3 = tmp_path / "c.txt"
    mpm.tune_cache_save(str(f3))
    mpm.tune_cache_load(str(f3))
    assert mpm.tune_cache_lookup(3, 1_000_000, 32768, 152) == SHAPES


@pytest.mark.parametrize("body", [
    "gbmpm-tune 2\n",                                       # other version
    "gbmpm-tune 1\n2 10 6 132 2 256 16 128 8 256\n",        # short line
    "gbmpm-tune 1\n4 10 6 132 2 256 16 128 8 256 2 256\n",  # dimension 4
    "gbmpm-tune 1\n2 10 6 132 7 256 16 128 8 256 2 256\n",  # not a candidate
    "gbmpm-tune 1\n2 10 6 132 2 256 16 128 8 256 2 256 x\n",  # trailing text
])
def test_malformed_files_are_refused_whole(tmp_path, body):
    f = tmp_path / "bad.txt"
    f.write_text(body + "2 11 7 99 2 256 2 256 2 256 2 256\n")
    with pytest.raises(mpm.MPMError):
        mpm.tune_cache_load(str(f))
    assert mpm.tune_cache_lookup(2, 2048, 128, 99) is None  # nothing of a refused file is added


def test_missing_file_is_an_argument_error(tmp_path):
    with pytest.raises(mpm.MPMError):
        mpm.tune_cache_load(str(tmp_path / "none.txt"))


def test_tile_edge_lines_round_trip(tmp_path):
    """Tile-edge entries (from mpm_tune_tile_edge) are kept in the same file as lines
    "edge dim log2_particles log2_nodes sms tile_edge" and survive a save and a load."""
    f = tmp_path / "edge.txt"
    f.write_text("gbmpm-tune 1\nedge 2 10 14 132 8\nedge 2 14 14 132 4\n")
    mpm.tune_cache_load(str(f))
    g = tmp_path / "edge_out.txt"
    mpm.tune_cache_save(str(g))
    lines = g.read_text().splitlines()
    assert "edge 2 10 14 132 8" in lines and "edge 2 14 14 132 4" in lines


@pytest.mark.parametrize("line", [
    "edge 3 10 14 132 8",      # 3D has one tile shape
    "edge 2 10 14 132 6",      # not an edge
    "edge 2 10 14 132",        # short
    "edge 2 10 14 0 4",        # no SMs
    "edge 2 10 14 132 8 x",    # trailing text
])
def test_malformed_tile_edge_lines_are_refused_whole(tmp_path, line):
    f = tmp_path / "bad_edge.txt"
    f.write_text("gbmpm-tune 1\n" + line + "\n2 12 7 98 2 256 2 256 2 256 2 256\n")
    with pytest.raises(mpm.MPMError):
        mpm.tune_cache_load(str(f))
    assert mpm.tune_cache_lookup(2, 4096, 128, 98) is None
