"""The bench's oracle-error summary (CPU): the per-pixel error relative to
|I_ref| + 1e-3 max(I_ref), the tolerance by storage, and the flux error."""
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
