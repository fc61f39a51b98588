"""Host-side logic of bench.py that needs no GPU: the DRAM-traffic record is keyed on the
bulk kernel's own source, so edits elsewhere in the library keep it and edits to the kernel
drop it (the bench then reports traffic as null until it is measured again)."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_traffic_record_keyed_on_bulk_kernel_source(tmp_path, monkeypatch):
    import bench

    csrc = os.path.join(ROOT, "paper_1409_5929_gb300", "csrc")
    dst = tmp_path / "paper_1409_5929_gb300" / "csrc"
    shutil.copytree(csrc, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._kernel_hash()
    src = (dst / "lbm.cu").read_text()
    marker = "__global__ void k_wall("
    assert src.count(marker) == 1
    cut = src.rindex("template <", 0, src.index(marker))
    (dst / "lbm.cu").write_text(src + "\n// a later host-side edit\n")
    assert bench._kernel_hash() == h0
    (dst / "lbm.cu").write_text(src[:cut] + "// an edit of the bulk kernel\n" + src[cut:])
    assert bench._kernel_hash() != h0
    (dst / "lbm.cu").write_text(src)
    (dst / "lbm_physics.cuh").write_text((dst / "lbm_physics.cuh").read_text() + "\n")
    assert bench._kernel_hash() != h0
    monkeypatch.setattr(bench, "ROOT", ROOT)
    rec = bench.TRAFFIC[("f32", bench.NR, bench.NZ)]
    assert len(rec[0]) == 16 and rec[1] > 0
