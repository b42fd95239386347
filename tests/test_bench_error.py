"""The bench's host logic (CPU): the oracle-error summary (the per-pixel error
relative to |I_ref| + 1e-3 max(I_ref), the tolerance by storage, and the flux
error), the launch and layout strings, the use of a committed profile's
traffic, and the roofline fraction."""
import numpy as np

import bench


def test_oracle_error_summary():
    ref = np.array([1.0, 2.0, 0.0, 4.0])
    gpu = np.array([1.0 + 1e-6, 2.0, 4e-9, 4.0 - 8e-5])
    e = bench.oracle_error([(ref[:2], gpu[:2]), (ref[2:], gpu[2:])], "f32")
    assert e["pixels"] == 4 and e["tolerance"] == 1e-5
    # worst pixel: 8e-5 / (4 + 4e-3), reported to three significant digits
    assert abs(e["max_rel"] / (8e-5 / 4.004) - 1.0) < 1e-2
    # 4e-9 against the floor 4e-3 is 1e-6: within; 8e-5 / 4.004 is not
    assert e["within_tolerance"] == 0.75
    assert abs(e["flux_rel"] / (abs(gpu.sum() - ref.sum()) / ref.sum()) - 1.0) < 1e-2
    assert bench.oracle_error([(ref, gpu)], "bf16")["tolerance"] == 1e-2
    assert bench.oracle_error([(ref, gpu)], "bf16")["within_tolerance"] == 1.0


def test_launch_and_layout_specs():
    """The bench's launch and layout strings: fields in order, optional ones 0."""
    L = bench.parse_launch("4,8,4,2,1,64")
    assert L == {"packet": (4, 8), "cta_warps": 4, "depth": 2, "persistent": 0, "regcap": 1, "region": 64, "group": 0}
    L = bench.parse_launch("8,4,8,4,1,0,4")
    assert L["persistent"] == 1 and L["region"] == 0 and L["group"] == 4
    assert bench.parse_layout("8,4,0") == [8, 4, 0, 0]
    assert bench.parse_layout("4,4,1,1") == [4, 4, 1, 1]
    assert list(bench.parse_layout("")) == [0, 0, 0, 0]
    for spec in bench.PINNED.values():  # every pinned entry parses
        bench.parse_launch(spec[0])
        assert len(bench.parse_layout(spec[1])) == 4


def test_recorded_traffic_matches_source_launch_and_layout(tmp_path, monkeypatch):
    """A profile's traffic is used only for the kernel source it was taken on
    and the launch and layout it names."""
    import hashlib
    src = tmp_path / "paper_2609_09322_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "march.cu").write_bytes(b"// kernel source\n")
    digest = hashlib.sha256(b"// kernel source\n").hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "march_demo.md").write_text(
        f"march.cu sha256[:16]: {digest}\n\ntimed configuration: --launch 4,8,4,2,1,64 --layout 8,4,0\n\n"
        "traffic_bytes_per_launch: 2.5e+10\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    launch, layout = bench.parse_launch("4,8,4,2,1,64"), bench.parse_layout("8,4,0")
    assert bench.recorded_traffic("demo", launch, layout) == 2.5e10
    assert bench.recorded_traffic("demo", bench.parse_launch("4,8,8,2,1,64"), layout) is None
    assert bench.recorded_traffic("demo", launch, bench.parse_layout("8,4,0,1")) is None
    assert bench.recorded_traffic("absent", launch, layout) is None
    (src / "march.cu").write_bytes(b"// kernel source, changed\n")
    assert bench.recorded_traffic("demo", launch, layout) is None


def test_committed_profiles_name_the_pinned_configurations():
    """Each committed march profile names the launch and layout that the
    bench pins for its workload."""
    import os
    import re
    for tag, pin in (("batched", "batched"), ("time_delay", "time_delay"), ("time_delay_bf16", "time_delay_bf16"),
                     ("precision", "precision")):
        text = open(os.path.join(bench.ROOT, "profiles", f"march_{tag}.md")).read()
        m = re.search(r"timed configuration:\s*--launch\s+(\S+)\s+--layout\s+(\S+)", text)
        assert m, tag
        assert bench.parse_launch(m.group(1)) == bench.parse_launch(bench.PINNED[pin][0]), tag
        assert bench.parse_layout(m.group(2)) == bench.parse_layout(bench.PINNED[pin][1]), tag
        assert re.search(r"traffic_bytes_per_launch:\s*[0-9.eE+]+", text), tag


def test_roofline_fraction():
    r = bench.roofline(samples=10**9, bytes_per_sample=32, kernel_ms=10.0, traffic=1e9, compulsory=5e8)
    assert abs(r["achieved"] - 3200.0) < 1e-6
    assert abs(r["frac"] - round(3200.0 / r["peak"], 4)) < 1e-9
    assert r["traffic"] == 1e9 and r["bytes_per_sample"] == 32
