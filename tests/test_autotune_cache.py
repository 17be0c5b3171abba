"""Host logic of the launch-shape autotuner's cache (no device needed): keys
separate devices, leaf sizes, leaf methods and tree shapes; a missing or
unreadable cache gives the library default."""
import json

from paper_2212_09562_b300 import autotune as A
from paper_2212_09562_b300 import mphf as M


def test_cache_keys_and_lookups(tmp_path, monkeypatch):
    monkeypatch.setenv("MPHF_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(A, "_device_name", lambda: "B300")
    assert A.tuned(16) == A.DEFAULT  # no cache file
    (tmp_path / "tune.json").write_text("not json")
    assert A.tuned(16) == A.DEFAULT  # unreadable cache
    keys = {A._key(16, True), A._key(16, M.PLAIN), A._key(16, M.SHOCKHASH), A._key(12, True),
            A._key(16, True, M.TREE_FANOUT2)}
    assert len(keys) == 5
    assert A._key(16, True) == "B300|l=16|rot=1"  # the RecSplit tree keeps the plain key
    data = {A._key(16, True): {"threads": 512, "blocks_per_sm": 2, "seeds_per_thread": 4},
            A._key(24, M.SHOCKHASH, M.TREE_FANOUT2): {"threads": 256, "blocks_per_sm": 0}}
    (tmp_path / "tune.json").write_text(json.dumps(data))
    assert A.tuned(16, True) == (512, 2, 4)
    assert A.tuned(16, True, M.TREE_FANOUT2) == A.DEFAULT
    assert A.tuned(24, M.SHOCKHASH, M.TREE_FANOUT2) == (256, 0, 0)  # an entry without the field
    assert A.tuned(24, M.SHOCKHASH) == A.DEFAULT
    monkeypatch.setattr(A, "_device_name", lambda: "another GPU")
    assert A.tuned(16, True) == A.DEFAULT
