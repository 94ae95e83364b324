"""Host logic of the autotuner (no GPU): which candidates a graph admits, the
cache key, and that a cached choice is returned without timing anything."""
import json

from paper_2510_21105_gb300 import autotune
from paper_2510_21105_gb300 import workloads as wl


def test_feasible_by_degree_and_size():
    small = wl.gnp(60, 0.1, seed=1)
    assert all(autotune.feasible(small, c) for c in autotune.CANDIDATES)
    dense = wl.gnp(300, 0.6, seed=2)   # max degree above 127: only the int16 layout
    assert dense.maxdeg > 127
    ok = [c for c in autotune.CANDIDATES if autotune.feasible(dense, c)]
    assert ok and all(c.get("variant") == 0 and c.get("field_bits") == 16 for c in ok)
    big = wl.gnm(33000, 40000, seed=3)  # beyond the packed layout's uint16 positions with a sign bit
    assert not autotune.feasible(big, dict(variant=0, field_bits=7, threads_per_cta=128))
    assert autotune.feasible(big, dict(variant=1))


def test_candidates_are_distinct():
    keys = [json.dumps(c, sort_keys=True) for c in autotune.CANDIDATES]
    assert len(keys) == len(set(keys))


def test_shape_key_and_cache_hit(tmp_path):
    g = wl.torus(10, seed=4)
    key = autotune.shape_key(g, 4096, 4)
    assert key == f"n{g.n}_m{g.m}_d{g.maxdeg}_w1_R4096_S4"
    cache = tmp_path / "cache.json"
    cache.write_text(json.dumps({key + "_saturated": {"opts": {"variant": 1}, "times": {"0": 1.5}}}))
    opts, times = autotune.tune(g, wl.linear_betas(0.1, 1.0, 8), 4096, 4, cache_path=str(cache),
                                context="saturated")
    assert opts == {"variant": 1} and times == {"0": 1.5}


def test_saturated_context_drops_pairs_and_splits():
    """Saturated: no CTA-pair kernel, and the one-CTA multi-spin-coded layout
    runs every word in one kernel (msc_no_split); alone: the candidates as
    listed."""
    g = wl.gnp(60, 0.1, seed=1)
    alone = autotune.candidates_for(g, "alone")
    sat = autotune.candidates_for(g, "saturated")
    assert alone == [c for c in autotune.CANDIDATES if autotune.feasible(g, c)]
    assert all(c.get("variant") != 3 for c in sat)
    assert [c for c in sat if c.get("variant") == 1] == [dict(variant=1, msc_no_split=1)]
    assert [c for c in sat if c.get("variant") == 0] == [c for c in alone if c.get("variant") == 0]
