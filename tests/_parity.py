"""Shared helpers for the GPU parity tests: tolerances and storage roundings
that build "what the GPU stores" inputs for the oracle, written here from the
storage formats' definitions (independently of the library's pack kernel)."""
import numpy as np

# FP32 path: 1e-5 relative per pixel, with an absolute floor of 1e-5 * 1e-3 of
# the image maximum for near-empty pixels.
FP32_REL = 1e-5
FLOOR_FRAC = 1e-3


def parity_report(gpu, ref, rel=FP32_REL, floor_frac=FLOOR_FRAC):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    peak = float(np.abs(ref).max()) if ref.size else 0.0
    tol = rel * np.abs(ref) + rel * floor_frac * peak
    err = np.abs(gpu - ref)
    bad = err > tol
    bright = np.abs(ref) > floor_frac * peak
    worst_rel = float((err[bright] / np.abs(ref[bright])).max()) if bright.any() else 0.0
    return dict(n_bad=int(bad.sum()), n=int(ref.size), worst_rel=worst_rel,
                worst_abs=float(err.max()) if err.size else 0.0, peak=peak)


def assert_parity(gpu, ref, rel=FP32_REL, floor_frac=FLOOR_FRAC, what=""):
    r = parity_report(gpu, ref, rel, floor_frac)
    assert r["n_bad"] == 0, f"{what}: {r['n_bad']}/{r['n']} pixels beyond tolerance {rel}: {r}"
    return r


def bf16_round(x) -> np.ndarray:
    """float -> float32 (nearest) -> bfloat16 (nearest, ties to even), as float32."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (u & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).reshape(f.shape)


def four_velocity_f16(beta) -> np.ndarray:
    """u = Gamma beta from float64 arithmetic ((bx^2 + by^2) + bz^2, 1/sqrt(1 - b2),
    beta * Gamma), rounded once to float16."""
    b = np.asarray(beta, dtype=np.float64)
    b2 = (b[..., 0] * b[..., 0] + b[..., 1] * b[..., 1]) + b[..., 2] * b[..., 2]
    g = 1.0 / np.sqrt(1.0 - b2)
    return (b * g[..., None]).astype(np.float16)


def beta_from_u(u) -> np.ndarray:
    """beta = u / sqrt(1 + |u|^2) in float64: the velocity the BF16/F16 record encodes."""
    u = np.asarray(u, dtype=np.float64)
    uu = (u * u).sum(axis=-1)
    return u / np.sqrt(1.0 + uu)[..., None]
