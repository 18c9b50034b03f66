"""The persisted launch-shape file (HN_TUNE_CACHE, the runtime configuration file of Sec. 3):
host-side store and lookup through the C ABI, no GPU."""
import pytest


@pytest.fixture(scope="module")
def hn():
    import __graft_entry__ as g
    g.build()
    from paper_0904_4152_gb300 import hn
    return hn


def test_missing_file_has_no_entry(hn, tmp_path):
    assert hn.hn_tune_cache_lookup(str(tmp_path / "none"), "NVIDIA GB300", 10, 1, 0, 0, 2) is None


def test_store_then_lookup_round_trip(hn, tmp_path):
    path = str(tmp_path / "tune.txt")
    a = (7, 16, 2, 0, 1, 0, 0, 1)
    b = (5, 4, 1, 1, 0, 1, 10, 0)
    hn.hn_tune_cache_store(path, "NVIDIA GB300", 10, 1, 0, 0, 2, a)
    hn.hn_tune_cache_store(path, "NVIDIA GB300", 12, 2, 1, 1, 3, b)
    assert hn.hn_tune_cache_lookup(path, "NVIDIA GB300", 10, 1, 0, 0, 2) == a
    assert hn.hn_tune_cache_lookup(path, "NVIDIA GB300", 12, 2, 1, 1, 3) == b
    # every field of the key counts
    for key in [("NVIDIA B200", 10, 1, 0, 0, 2), ("NVIDIA GB300", 11, 1, 0, 0, 2),
                ("NVIDIA GB300", 10, 0, 0, 0, 2), ("NVIDIA GB300", 10, 1, 1, 0, 2),
                ("NVIDIA GB300", 10, 1, 0, 1, 2), ("NVIDIA GB300", 10, 1, 0, 0, 3)]:
        assert hn.hn_tune_cache_lookup(path, *key) is None, key


def test_store_replaces_the_entry_of_its_key(hn, tmp_path):
    path = str(tmp_path / "tune.txt")
    hn.hn_tune_cache_store(path, "GPU", 9, 0, 0, 0, 2, (6, 16, 2, 0, 1, 0, 0, 0))
    hn.hn_tune_cache_store(path, "GPU", 8, 0, 0, 0, 2, (4, 2, 2, 0, 1, 0, 0, 1))
    hn.hn_tune_cache_store(path, "GPU", 9, 0, 0, 0, 2, (3, 1, 0, 0, 0, 0, 9, 0))
    lines = open(path).read().splitlines()
    assert len(lines) == 2
    assert hn.hn_tune_cache_lookup(path, "GPU", 9, 0, 0, 0, 2) == (3, 1, 0, 0, 0, 0, 9, 0)
    assert hn.hn_tune_cache_lookup(path, "GPU", 8, 0, 0, 0, 2) == (4, 2, 2, 0, 1, 0, 0, 1)


def test_malformed_and_out_of_range_lines_are_ignored(hn, tmp_path):
    path = tmp_path / "tune.txt"
    path.write_text("# comment\n"
                    "GPU|10|1|0|0|2 7 16 2 0 1 0 0 1\n"
                    "GPU|10|1|0|0|2 7 3 2 0 1 0 0 0\n"          # cluster 3: out of range
                    "GPU|11|1|0|0|2 7 16\n"                      # too few fields
                    "GPU|12|1|0|0|2 7 16 2 0 1 0 0 3\n"          # sweep 3: out of range
                    "GPU|13|1|0|0|2 7 16 2 0 1 0 0 1 5\n"        # a field too many
                    "GPU|14|1|0|0|2 7 16 2 0 1 0 0 x\n"          # not a number
                    "GPU|15|1|0|0|2 6 8 2 0 1 0 0\n"             # no sweep field: sweep 0
                    "garbage line\n")
    assert hn.hn_tune_cache_lookup(str(path), "GPU", 10, 1, 0, 0, 2) == (7, 16, 2, 0, 1, 0, 0, 1)
    for L in (11, 12, 13, 14):
        assert hn.hn_tune_cache_lookup(str(path), "GPU", L, 1, 0, 0, 2) is None, L
    assert hn.hn_tune_cache_lookup(str(path), "GPU", 15, 1, 0, 0, 2) == (6, 8, 2, 0, 1, 0, 0, 0)
    # a store keeps the other lines as they are
    hn.hn_tune_cache_store(str(path), "GPU", 16, 1, 0, 0, 2, (8, 16, 2, 0, 1, 0, 0, 0))
    text = path.read_text()
    assert "garbage line" in text and "# comment" in text


def test_out_of_range_shapes_and_separators(hn, tmp_path):
    path = str(tmp_path / "tune.txt")
    with pytest.raises(hn.HnError) as e:
        hn.hn_tune_cache_store(path, "GPU", 10, 1, 0, 0, 2, (7, 5, 2, 0, 1, 0, 0, 0))
    assert e.value.status == hn.HN_ERR_ARG
    with pytest.raises(hn.HnError) as e:
        hn.hn_tune_cache_store(path, "GPU", 10, 1, 0, 0, 2, (7, 16, 2, 0, 1, 0, 0, 3))
    assert e.value.status == hn.HN_ERR_ARG
    # a separator inside the GPU name cannot split the key
    hn.hn_tune_cache_store(path, "odd|name", 10, 1, 0, 0, 2, (7, 16, 2, 0, 1, 0, 0))   # sweep 0
    assert hn.hn_tune_cache_lookup(path, "odd|name", 10, 1, 0, 0, 2) == (7, 16, 2, 0, 1, 0, 0, 0)
    assert hn.hn_tune_cache_lookup(path, "odd", 10, 1, 0, 0, 2) is None
