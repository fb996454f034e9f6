"""Tile autotuner: cache keys and storage (CPU), timed search and use of the
tuned shapes (GPU)."""
import json
import os

import numpy as np
import pytest

from paper_2305_05988_gb300 import autotune


def test_size_bucket_and_key():
    assert autotune.size_bucket((100, 90)) == 128
    assert autotune.size_bucket((16, 16, 16)) == 16
    assert autotune.size_bucket((22,)) == 16 and autotune.size_bucket((23,)) == 32  # geometric midpoint 22.6
    k = autotune.tune_key("GB300", "cg", "laplacian", (256, 256, 256), "f64", "grid")
    assert k == "GB300|cg|laplacian|3d|n256|f64|teamgrid"


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cache(path) == {}
    autotune.save_cache({"a": {"tile_rows": 8, "tile_planes": 16}}, path)
    assert json.load(open(path))["a"]["tile_planes"] == 16
    assert autotune.load_cache(path)["a"]["tile_rows"] == 8


@pytest.mark.gpu
def test_tune_picks_a_candidate_and_tuned_tiles_solve_the_same_system(tmp_path):
    torch = pytest.importorskip("torch")
    import paper_2305_05988_gb300 as hs
    from paper_2305_05988_gb300 import inputs
    path = str(tmp_path / "tune.json")
    shape = (48, 40, 36)
    e = autotune.tune(shape, "laplacian", "cg", "grid", path=path, iters=10, planes=(0, 8, 32))
    assert e["tile_rows"] in (4, 8, 16) and e["tile_planes"] in (0, 8, 32)
    assert len(e["trials"]) == 9 and all(t["ms_per_iter"] > 0 for t in e["trials"])
    assert autotune.lookup(shape, "laplacian", "cg", "grid", path=path)["tile_rows"] == e["tile_rows"]
    A = hs.Operator.laplacian(shape)
    b = torch.from_numpy(inputs.rhs_uniform(shape, 3)).cuda()
    x0, i0 = hs.cg(A, b, tol=1e-10)
    x1, i1 = hs.cg(A, b, tol=1e-10, tile_rows=e["tile_rows"], tile_planes=e["tile_planes"])
    x2, i2 = hs.cg(A, b, tol=1e-10, max_blocks=1, tile_rows=16, tile_planes=8)
    for x, i in ((x1, i1), (x2, i2)):
        assert i.status == "OK" and abs(i.iters - i0.iters) <= 2
        assert (torch.linalg.norm(x - x0) / torch.linalg.norm(x0)).item() <= 1e-8


@pytest.mark.gpu
def test_batch_uses_autotuned_planes(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    import oracle
    import paper_2305_05988_gb300 as hs
    from paper_2305_05988_gb300 import inputs
    monkeypatch.setenv("HSOLVE_TUNE_CACHE", str(tmp_path / "tune.json"))
    shapes = [(12, 12, 12), (20, 20, 20), (30, 30), (9, 9, 9)]
    ops = [hs.Operator.laplacian(s) for s in shapes]
    batch = hs.Batch(ops, ["cg"] * 4, autotune=True)
    assert len(batch.tile_planes) == 4 and os.path.exists(str(tmp_path / "tune.json"))
    bs = [torch.from_numpy(inputs.uniform_pm1(4, 7, int(np.prod(s)))).cuda() for s in shapes]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        xs, infos = batch.solve(bs, tol=1e-8)
    st.synchronize()
    for s, b, x, i in zip(shapes, bs, xs, infos):
        assert i.status == "OK"
        assert oracle.Operator(s).relres(b.cpu().numpy(), x.cpu().numpy()) <= 1.5e-8
