"""SpMV autotuner: the choice per stored operator (format and threads per block) is visible through
bgs_level_format, is written to the file named by BGS_AUTOTUNE_CACHE, and a later process obeys that
file (here rewritten so that every operator uses CSR with one thread per row at 256 threads per
block, then so that the full operator uses the node-block layout) and still solves to the same
answer, the full operator's product matching the oracle's."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
import battery_system as bs
import paper_2602_13079_gb300 as bgs
system = bs.assemble(grid=bs.Grid(3, 24, 20, 18), seed=11)
out = {}
for precision in (0, 1):
    g = bgs.solver_for_system(system, device=False, precision=precision, max_coarse=40)
    g.bgs_setup()
    fmt = []
    for k in range(5):
        L = g.bgs_num_levels(k)
        for l in range(L - 1):    # the coarsest level is solved through its dense inverse
            fmt += [list(g.bgs_level_format(k, l, w, with_block=True)) for w in (0, 1, 2)]
    xin = torch.tensor(np.random.default_rng(5).standard_normal(system.ndof), dtype=torch.float64, device="cuda")
    y = torch.zeros(system.ndof, dtype=torch.float64, device="cuda")
    g.bgs_full_spmv(xin, y)
    torch.cuda.synchronize()
    x = np.zeros(system.ndof)
    info = g.bgs_solve(system.b, x)
    out[precision] = {"fmt": fmt, "full": list(g.bgs_level_format(0, 0, 3, with_block=True)),
                      "spmv": y.cpu().numpy().tolist(),
                      "iters": info.iters, "converged": bool(info.converged), "x": x.tolist()}
    g.close()
json.dump(out, open(sys.argv[1], "w"))
"""


def _oracle_spmv():
    import battery_system as bs
    import oracle
    system = bs.assemble(grid=bs.Grid(3, 24, 20, 18), seed=11)
    x = np.random.default_rng(5).standard_normal(system.ndof)
    return oracle.bgs_for_system(system, setup=False).full_matvec(x)


def _run(tmp_path, cache, tag):
    res = tmp_path / f"{tag}.json"
    env = dict(os.environ, BGS_AUTOTUNE_CACHE=str(cache), PYTHONPATH=ROOT)
    subprocess.run([sys.executable, "-c", CHILD, str(res)], cwd=ROOT, env=env, check=True, timeout=600)
    return json.loads(res.read_text())


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_13079_gb300 import _build
    _build.build()


def test_autotune_cache_written_and_obeyed(built, tmp_path):
    cache = tmp_path / "tune.txt"
    first = _run(tmp_path, cache, "first")
    lines = [ln.split() for ln in cache.read_text().splitlines() if ln.strip()]
    assert lines and all(len(f) == 6 for f in lines)
    for p in ("0", "1"):
        assert first[p]["converged"]
        assert all(f >= -1 and t in (128, 256, 512) for f, t in first[p]["fmt"])
    # a second process with the same file times nothing new and makes the same choices
    again = _run(tmp_path, cache, "again")
    assert len(cache.read_text().splitlines()) == len(lines)
    for p in ("0", "1"):
        assert again[p]["fmt"] == first[p]["fmt"]
        assert again[p]["x"] == first[p]["x"]          # same kernels, same order: bit-identical
    # force CSR with one thread per row at 256 threads per block everywhere (choice code 9: CSR with
    # 2^(2 - 2) lanes, block-size code 1)
    cache.write_text("".join(" ".join(f[:5] + ["9"]) + "\n" for f in lines))
    forced = _run(tmp_path, cache, "forced")
    for p in ("0", "1"):
        assert forced[p]["converged"]
        assert all(f == 1 and t == 256 for f, t in forced[p]["fmt"])
        x0, x1 = np.array(first[p]["x"]), np.array(forced[p]["x"])
        assert np.linalg.norm(x1 - x0) <= 1e-6 * np.linalg.norm(x0)


def test_node_block_layout_for_the_full_operator(built, tmp_path):
    cache = tmp_path / "tune.txt"
    first = _run(tmp_path, cache, "first")
    lines = [ln.split() for ln in cache.read_text().splitlines() if ln.strip()]
    ndof = str(43200)
    full = [f for f in lines if f[0] == ndof and f[1] == ndof and f[3] == "8" and f[4] == "1"]
    assert len(full) == 1                          # the full operator, FP64, timed as a plain product
    # choice code 33: node blocks (format code 8) at 256 threads per block
    cache.write_text("".join(" ".join(f[:5] + ["33"] if f in full else f) + "\n" for f in lines))
    forced = _run(tmp_path, cache, "bsr")
    ref = _oracle_spmv()
    for p in ("0", "1"):
        assert forced[p]["full"] == [-2, 256]
        assert forced[p]["converged"]
        y = np.array(forced[p]["spmv"])
        # the same products, summed block by block: rounding differences only
        assert np.allclose(y, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
        x0, x1 = np.array(first[p]["x"]), np.array(forced[p]["x"])
        assert np.linalg.norm(x1 - x0) <= 1e-6 * np.linalg.norm(x0)
        assert abs(forced[p]["iters"] - first[p]["iters"]) <= 1
