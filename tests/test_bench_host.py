"""Host-side logic of bench.py: algorithmic bytes, the traffic table's source
check, and the serving sample (CPU only)."""
import os
import shutil

import pytest

import bench
from paper_1908_05834_gb300 import inputs


def test_algorithmic_bytes_per_stage():
    nc, nnz = 1000, 3500
    # update: 12 B per entry; pointer, c_in, c_out, |K|_phi per cell
    assert bench.algorithmic_bytes("update", nc, nnz) == nnz * 12 + nc * 32
    assert bench.algorithmic_bytes("update", nc, nnz, c_bytes=4) == nnz * 12 + nc * 24
    # one column and one row pass
    assert bench.algorithmic_bytes("scaling", nc, nnz) == 2 * (nnz * 12 + nc * 32)
    # both views of the entries, 2 n_c constraint nodes
    assert bench.algorithmic_bytes("cg_matvec", nc, nnz) == 2 * nnz * 12 + 2 * nc * 32
    assert bench.algorithmic_bytes("smooth", nc, nnz) == 2 * nnz * 12 + 2 * nc * 48
    with pytest.raises(KeyError):
        bench.algorithmic_bytes("assemble", nc, nnz)


def test_traffic_is_reported_only_for_the_source_it_was_measured_on(tmp_path, monkeypatch):
    got, line = bench.measured_traffic("k_cg_matvec", "vortex2d_1024")
    assert got is not None and got > 0 and "k_cg_matvec" in line
    assert bench.measured_traffic("k_cg_matvec", "deform3d_128") == (None, None)
    assert bench.measured_traffic("k_assemble", "vortex2d_1024") == (None, None)
    # a copy of the sources with the kernel's body changed: its line no longer applies
    csrc = tmp_path / "csrc"
    shutil.copytree(bench.CSRC, csrc)
    text = (csrc / "sparse.cu").read_text()
    head = "__global__ void __launch_bounds__(kTileThreads) k_cg_matvec("
    assert head in text
    (csrc / "sparse.cu").write_text(text.replace("const double acc = block_sum(er.acc + ec.acc);",
                                                 "const double acc = block_sum(ec.acc + er.acc);"))
    before = bench.kernel_source_hash("k_cg_matvec")
    monkeypatch.setattr(bench, "CSRC", str(csrc))
    assert bench.kernel_source_hash("k_cg_matvec") != before
    assert bench.measured_traffic("k_cg_matvec", "vortex2d_1024") == (None, None)
    # the other kernels' lines still apply
    assert bench.measured_traffic("k_spmv", "vortex2d_1024")[0] is not None


def test_serving_sample_is_bounded_and_keeps_the_stream_order():
    picked = bench._serving_sample(inputs, 6, 150000, 3)
    assert len(picked) == 6
    stream = inputs.serving_requests(512)
    small = [r for r in stream if r.nc <= 150000][:6]
    assert [r.rid for r in picked] == [r.rid for r in small]
    assert all(r.nc <= 150000 and r.steps == min(3, s.steps) for r, s in zip(picked, small))
