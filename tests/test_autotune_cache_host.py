"""The autotuner's JSON decision cache (host logic, no GPU): keys are
order-independent in the image list and separate GPUs, budgets and
candidate sets; the file survives concurrent-looking rewrites and a
corrupt file reads as empty."""
import json

from paper_2604_21984_gb300 import batch


def test_key_is_canonical_and_discriminating():
    k = lambda sizes, **kw: batch.tune_key(sizes, kw.get("iters", 100), kw.get("cands", ((16, 4), (8, 4))),
                                           0.05, 0.06, kw.get("gpu", "GB300"))
    a = k([(512, 768), (256, 256)])
    assert a == k([(256, 256), (512, 768)])                 # order of the images does not matter
    assert a != k([(512, 768), (256, 256)], iters=500)
    assert a != k([(512, 768), (256, 256)], gpu="other")
    assert a != k([(512, 768), (256, 256)], cands=((16, 4),))
    assert a != k([(512, 768), (256, 257)])
    assert json.loads(a)["images"] == [[256, 256], [512, 768]]


def test_store_and_load(tmp_path):
    p = str(tmp_path / "tune.json")
    assert batch.cache_load(p, "x") is None                  # no file yet
    batch.cache_store(p, "x", {"pick": [16, 4], "table": [[16, 4, 3.5, 33.5]]})
    batch.cache_store(p, "y", {"pick": [8, 2], "table": []})
    assert batch.cache_load(p, "x")["pick"] == [16, 4]
    assert batch.cache_load(p, "y")["pick"] == [8, 2]
    with open(p, "w") as f:
        f.write("{not json")
    assert batch.cache_load(p, "x") is None                  # corrupt file: empty cache
    batch.cache_store(p, "z", {"pick": [8, 4], "table": []})
    assert batch.cache_load(p, "z")["pick"] == [8, 4]
