"""Host logic of bench.py that needs no GPU: the source hash that ties the
committed ncu DRAM-traffic figures to the stencil sources they were taken
with, and the parsing of those figures."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _closure(units):
    csrc = os.path.join(ROOT, "paper_2407_00041_gb300", "csrc")
    seen, todo = set(), list(units)
    while todo:
        f = todo.pop()
        if f in seen or not os.path.exists(os.path.join(csrc, f)):
            continue
        seen.add(f)
        todo += re.findall(r'^\s*#\s*include\s+"([^"]+)"', open(os.path.join(csrc, f)).read(), flags=re.M)
    return seen


def test_source_hash_covers_the_stencil_units_and_their_headers():
    files = _closure(("dd_hop_f32.cu", "dd_hop_f16.cu"))
    assert {"dd_hop_f32.cu", "dd_hop_f16.cu", "dd_hop.cuh", "dd_device.cuh", "dd_ops.h"} <= files
    assert "dd_hop_pair.cuh" not in files  # the paired stencil is not part of these launches
    h = bench.kernel_source_hash()
    assert re.fullmatch(r"[0-9a-f]{16}", h)
    assert h == bench.kernel_source_hash(("dd_hop_f16.cu", "dd_hop_f32.cu"))  # order-independent


def test_profile_traffic_is_read_only_for_the_current_sources(tmp_path, monkeypatch):
    for prec in ("f32", "f16"):
        path = os.path.join(ROOT, "profiles", f"dslash_{prec}_48x48x48x96.md")
        txt = open(path).read()
        m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
        assert m and float(m.group(1)) > 1e9
        # a profile recorded with other sources gives no traffic figure
        fake = tmp_path / "profiles"
        fake.mkdir(exist_ok=True)
        pkg = tmp_path / "paper_2407_00041_gb300"
        if not pkg.exists():  # the same sources, so only the recorded hash differs
            pkg.symlink_to(os.path.join(ROOT, "paper_2407_00041_gb300"), target_is_directory=True)
        (fake / f"dslash_{prec}_48x48x48x96.md").write_text(
            re.sub(r"kernel_sources_sha256_16:\s*[0-9a-f]+", "kernel_sources_sha256_16: 0000000000000000", txt))
        real = bench.kernel_source_hash()
        monkeypatch.setattr(bench, "ROOT", str(tmp_path))
        assert bench.kernel_source_hash() == real  # the linked sources hash the same
        assert bench.profile_traffic(prec) is None
        monkeypatch.undo()
