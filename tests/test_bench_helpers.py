"""Host logic of bench.py that the measurement rests on (CPU only): the
strided sample the autotuner and the FP64 leg time, and the DRAM-traffic
record that is reported only while the kernel sources it was taken from are
unchanged."""
import hashlib
import os

import numpy as np
import pytest

import bench


def test_strided_sample_spreads_whole_blocks_over_every_part():
    torch = pytest.importorskip("torch")
    n = 100_000
    ids = np.arange(n, dtype=np.int64)
    rec = np.zeros((n, 64), dtype=np.uint8)
    rec[:, :8] = ids.view(np.uint8).reshape(n, 8)          # each record carries its index
    segs = torch.from_numpy(rec.reshape(-1))
    sub, m = bench.strided_sample(torch, segs, n, 20_000)
    got = sub.numpy().reshape(m, 64)[:, :8].copy().view(np.int64).ravel()
    assert m <= 20_000 and m % 32 == 0 and len(got) == m
    blocks = got.reshape(64, -1)                             # 64 blocks of consecutive steps
    assert blocks.shape[1] % 32 == 0
    assert np.all(np.diff(blocks, axis=1) == 1)
    starts = blocks[:, 0]
    assert starts[0] == 0 and starts[-1] + blocks.shape[1] == n   # first and last steps included
    gaps = np.diff(starts)
    assert gaps.max() - gaps.min() <= 1                      # evenly spread
    # a sample as large as the array is the array
    same, m2 = bench.strided_sample(torch, segs, n, n)
    assert m2 == n and same is segs


def _tree(tmp_path, src=b"kernel v1\n"):
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2309_15861_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cuh").write_bytes(src)
    h = hashlib.sha256(src).hexdigest()
    (tmp_path / "profiles" / "tracing_wl_traffic.txt").write_text(
        "# test record\nsteps 1000\ndram_bytes 85000\nbytes_per_step 85.0\nsha256 k.cuh " + h + "\n")
    return csrc / "k.cuh"


def test_recorded_traffic_is_reported_only_for_the_sources_it_was_taken_from(tmp_path, monkeypatch):
    f = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("wl", 2000) == pytest.approx(170000.0)   # scaled by the steps
    assert bench.recorded_traffic("other", 2000) is None                   # no record
    assert bench.traffic_record("wl") == {"bytes_per_step": 85.0, "current": True,
                                          "file": "profiles/tracing_wl_traffic.txt"}
    f.write_bytes(b"kernel v2\n")                                           # a kernel changed
    assert bench.recorded_traffic("wl", 2000) is None
    assert bench.traffic_record("wl")["current"] is False                   # the figure, marked stale
    os.remove(f)                                                            # or is gone
    assert bench.recorded_traffic("wl", 2000) is None
